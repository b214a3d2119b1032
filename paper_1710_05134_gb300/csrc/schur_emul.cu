// FP64-accurate Schur update on the tensor cores (the window flush of the front factorization).
//
// C(i, j) -= sum_c L(i, c) W(j, c), W = L D, for the pivots of one window (rank r <= 256).  GB300
// issues FP64 FMAs at about 1/64 of its FP32 rate, so the product is formed from bf16 pieces
// whose products the tensor cores sum exactly (an error-free splitting in the manner of Ozaki et
// al.):
//
//  * column balancing: column c of L is scaled by 2^{-u_c} and column c of W by 2^{u_c}, u_c half
//    the exponent of the pivot's magnitude with the sign reversed (max |W(., c)| is about
//    |D_c| max |L(., c)|), which leaves every product unchanged and keeps the spread of D out of
//    the rows;
//  * every row is scaled by a power of two 2^e with |x| < 2^{e-1} for all its entries, and
//    |x| 2^{8-e} (< 128) is written in balanced base-256 digits, sum_a d_a 256^{1-a}, a = 1..8,
//    d_1 in [0, 128], d_a in [-128, 127] otherwise, cut from the double's significand with integer
//    operations (the dropped tail is below 2^-63 of 2^e); each digit times the sign of x is exact
//    in bf16 and every digit product is at most 2^14 in magnitude;
//  * the tensor cores (tcgen05, accumulators in tensor memory) sum, for each level g = a + b
//    (2 <= g <= 9) and each half of the window (128 columns), the products s_a(i, c) t_b(j, c) in
//    one FP32 accumulator.  It holds at most 8 pairs x 128 columns x 2^14 = 2^24 in magnitude,
//    integers all along, so every FP32 sum is exact;
//  * the exact level sums of an entry are combined in integers and C(i, j) receives
//    -2^{e_i + f_j - 72} (V_hi 2^32 + V_lo), rounded once to FP64.
//
// The only roundings are the one FP64 product L D, the dropped digit tail and the final FP64
// conversion and subtraction: as accurate as an FP64 rank-r update.
//
// Tensor-core layout: a CTA owns a 128 x 32 tile of C (rows i, columns j).  Per 16-column step it
// issues eight MMAs, slice a of the L rows (M = 128) against slices 1 .. 9-a of the W rows stacked
// along N (N = 32 (9-a)), writing the accumulators of levels a+1 .. 9 side by side in tensor
// memory (8 levels x 32 columns per half window, two such buffers, so the MMAs of one half run
// while the epilogue reads the other); both operands are staged in shared memory by bulk copies
// in a five-step pipeline.
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>

#include "kep_tc.cuh"

namespace kep {

namespace {

constexpr int kSlices = 8;                    // digits of the FP64-accurate splitting
constexpr int kSlicesLow = 4;                 // digits of the reduced-precision splitting (KEP_SCHUR_FP32)
constexpr int kKB = kWindow / 8;              // 8-column blocks of a window
constexpr int kTM = 128;                      // tile rows (i): tensor-memory lanes
constexpr int kTN = 32;                       // tile columns (j) per digit of W
constexpr int kStages = 5;                    // shared-memory pipeline depth (16 columns each)
// per digit count S: one pipeline stage holds [k-block 2][slice S][row 128][16 B] of L digits and
// [k-block 2][slice S][row 32][16 B] of W digits; tensor memory holds 2 buffers x S level
// accumulators x 32 columns
template <int S>
struct Split {
  static constexpr uint32_t kStageA = 2 * S * kTM * 16;
  static constexpr uint32_t kStageB = 2 * S * kTN * 16;
  static constexpr uint32_t kStageBytes = kStageA + kStageB;
  static constexpr size_t kSmem = static_cast<size_t>(kStages) * kStageBytes + 1024;
  static constexpr uint32_t kTmemCols = 2 * S * kTN <= 256 ? 256u : 512u;
  static constexpr int kShift = 8 * (S + 1);  // 2^{e_i + f_j - kShift}: weight of the lowest level kept
};
constexpr int kEpiWarps = 16;                 // epilogue: warp w reads lanes 32 (w % 4), columns 8 (w / 4)
constexpr int kFlushThreads = (kEpiWarps + 2) * 32;   // + one copy warp, one MMA-issue warp
constexpr int kHalf = 8;                      // 16-column steps per accumulation (128 columns)
constexpr uint64_t kWaitNs = 2000000000ull;   // bounded waits: 2 s
// longest sleep between two tries of a wait, per role (the copy and MMA warps must react fast,
// the epilogue waits for a whole half window)
constexpr uint32_t kSleepCopy = 128, kSleepMma = 64, kSleepEpi = 1024;
constexpr int kNoExp = -(1 << 20);            // row maximum of an all-zero row

struct EmulArgs {
  __nv_bfloat16* Ls;   // digits of the balanced, scaled L rows, tile-contiguous (ldig_off)
  __nv_bfloat16* Ws;   // digits of the W rows (wdig_off)
  int32_t* eL;         // [R] row scale exponents
  int32_t* eW;
  int64_t R;           // rows of the digit arrays (a multiple of kTM, >= rows + kTM)
};

// Digit layouts: for the L rows, blocks of 128 rows, then 16-column steps, then the two 8-column
// halves, then the slice, then [128 rows][8 columns]; for the W rows the same with blocks of 32.
// One step of one tile is then a contiguous 32 KiB (L) and 8 KiB (W) run whose order is that of
// the shared-memory operands.
template <int S>
KEP_D int64_t ldig_off(int a, int32_t q, int64_t row) {      // q: 8-column block
  return (((((row >> 7) * (kWindow / 16) + (q >> 1)) * 2 + (q & 1)) * S + a) * kTM + (row & (kTM - 1))) * 8;
}
template <int S>
KEP_D int64_t wdig_off(int a, int32_t q, int64_t row) {
  return (((((row >> 5) * (kWindow / 16) + (q >> 1)) * 2 + (q & 1)) * S + a) * kTN + (row & (kTN - 1))) * 8;
}

KEP_HD int64_t digit_pitch(int64_t cap_rows) { return (cap_rows + kTM - 1) / kTM * kTM + kTM; }

// Workspace of one front (rows up to cap_rows): L digits, W digits, row exponents.
KEP_HD EmulArgs emul_args(void* ws, int64_t cap_rows) {
  EmulArgs E;
  E.R = digit_pitch(cap_rows);
  const int64_t plane = static_cast<int64_t>(kSlices) * kKB * E.R * 8;
  E.Ls = static_cast<__nv_bfloat16*>(ws);
  E.Ws = E.Ls + plane;
  E.eL = reinterpret_cast<int32_t*>(E.Ws + plane);
  E.eW = E.eL + E.R;
  return E;
}

// A batch of fronts on the tensor-core path: entries e0 .. e0 + nb - 1 of the level's batch
// arrays; entry e's workspace starts at ws + off[e] (bytes).
struct EmulBatch {
  unsigned char* ws;
  const int64_t* off;
  const int32_t* lf;    // the level's entries: front and shift (Batch)
  const int8_t* sh;
  int32_t e0, nb;
};
KEP_D int32_t emul_shift(const EmulBatch& B, int32_t b) { return B.sh ? B.sh[b] : 0; }
KEP_D EmulArgs entry_args(const EmulBatch& B, int32_t e, int64_t cap_rows) {
  return emul_args(B.ws + B.off[e], cap_rows);
}

KEP_D int bexp(double x) {                    // biased exponent field (0 for zero / subnormal)
  return static_cast<int>((__double_as_longlong(x) >> 52) & 0x7ff);
}

// W(i, c) = sum_c' L(i, c') D(c', c) for the window's pivot c (2x2 blocks mix two columns), from
// the window's pivot types and D entries cached in shared memory (column cl of the window, global
// column cg)
KEP_D double wval_s(const double* L, int64_t ld, int64_t i, int32_t cg, int32_t cl, const double* wself,
                    const double* woth, const int8_t* wpt) {
  const double x = L[static_cast<int64_t>(cg) * ld + i];
  const int8_t pt = wpt[cl];
  if (pt == 1) return x * wself[cl];
  if (pt == 2) return x * wself[cl] + L[static_cast<int64_t>(cg + 1) * ld + i] * woth[cl];
  return L[static_cast<int64_t>(cg - 1) * ld + i] * woth[cl] + x * wself[cl];
}

// Balancing shift of pivot column c: floor(-e/2) for the exponent e of its pivot's magnitude (the
// larger entry of a 2x2 block), 0 for a zero pivot.
KEP_D int balance_shift(const double* Dd, const double* De, const int8_t* pv, int32_t c) {
  const int8_t pt = pv[c];
  const double d = pt == 1 ? fabs(Dd[c])
                 : pt == 2 ? fmax(fabs(Dd[c]), fabs(De[c]))
                           : fmax(fabs(De[c - 1]), fabs(Dd[c]));
  const int e = bexp(d);
  if (e == 0) return 0;
  const int n = 1023 - e;
  return n >= 0 ? n / 2 : -((-n + 1) / 2);       // floor(n / 2)
}

// 64-bit fixed point floor(|x| 2^{-u} 2^{8-e} 2^56) of a normal double x (0 for zero/subnormal);
// below 2^63 when |x 2^-u| < 2^{e-1}.
KEP_D unsigned long long fixed64(double x, int u, int e) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bits >> 52) & 0x7ff);
  if (E == 0) return 0ull;
  const unsigned long long M = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = E - 1011 - u - e;             // value M 2^{E-1075} scaled by 2^{-u+8-e+56}
  if (sh >= 0) return M << sh;                 // sh <= 10 because the scaled value is below 2^63
  if (sh <= -64) return 0ull;
  return M >> (-sh);
}

// bf16 bit pattern of the integer d, |d| <= 128 (exact: at most 8 significant bits).  The float
// value comes from the magic-number construction (1.5 * 2^23 + d has unit spacing there, so the
// integer added to its bit pattern is exact, and subtracting 1.5 * 2^23 leaves d), two ALU/FMA-pipe
// operations instead of a conversion on the quarter-rate pipe.
KEP_D uint32_t digit_bits(int d) {
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// The leading S of the eight balanced digits of one value, times its sign, as bf16 bit patterns
// (S < 8 drops the rest: a truncation below 2^{-8S} of the row scale).
template <int S>
KEP_D void balanced_digits(double x, int u, int e, uint32_t (&d)[S]) {
  const unsigned long long Y = fixed64(x, u, e) + 0x0080808080808080ull;   // pre-carry of the low 7
  const bool neg = x < 0.0;
#pragma unroll
  for (int a = 0; a < S; ++a) {
    const int v = a == 0 ? static_cast<int>(Y >> 56) : static_cast<int>((Y >> (56 - 8 * a)) & 0xff) - 128;
    d[a] = digit_bits(neg ? -v : v);
  }
}

// The update a launch performs for batch entry b this step, false when there is none.  Window
// update (kWin): the pivots just accepted, columns [c0, c1) = [k, k + q), applied to the rest of
// the pivot window, columns [c1, we).  Flush: the window's pivots [ws, kend) applied to the
// trailing matrix, columns [we, m).  Rows [s, m) of L and rows [s, ce) of W take part, and C(i, j)
// is updated for j in [s, ce), i in [j, m).
template <bool kWin>
KEP_D bool emul_range(const LargeWork& W, int32_t b, int32_t m, int32_t& c0, int32_t& c1, int32_t& s, int32_t& ce) {
  if (W.done[b]) return false;
  if (kWin) {
    c0 = W.k[b];
    c1 = c0 + W.q[b];
    s = c1;
    ce = min(W.we[b], m);
  } else {
    if (!W.flush[b]) return false;
    c0 = W.ws[b];
    c1 = W.kend[b];
    s = W.we[b];
    ce = m;
  }
  return c1 > c0 && s < ce;
}

// Digits: per row, the scale exponents of the balanced L and W rows (W = L D formed on the fly),
// then the digits of every entry of the update's columns (zero up to the next multiple of 16
// columns).  A row is shared by NG threads (NG = 2, 4 or 8 from the update's width), thread g
// taking the 8-column blocks g, g + NG, ...; each 16-byte store holds one row's 8 digits of one
// slice and block, consecutive threads writing consecutive rows.
constexpr int kSThreads = 256;
template <bool kWin, int ND>
__global__ void __launch_bounds__(kSThreads) lf_slice_kernel(FrontTables T, SlotSet SS, LargeWork W, EmulBatch BA) {
  __shared__ int smx[2][kSThreads];
  __shared__ int su[kWindow];
  __shared__ double wself[kWindow], woth[kWindow];   // W = L D coefficients of the window's columns
  __shared__ int8_t wpt[kWindow];
  const int32_t b = BA.e0 + blockIdx.y;
  const int32_t t = BA.lf[b];
  const FactorSlot& S = SS.s[emul_shift(BA, b)];
  const EmulArgs E = entry_args(BA, blockIdx.y, T.m_alloc[t]);
  const int32_t m = T.m_sym[t] + S.d_in[t];
  int32_t c0, c1, s, ce;
  if (!emul_range<kWin>(W, b, m, c0, c1, s, ce)) return;
  const int32_t r = c1 - c0;
  const int64_t wrows = ce - s;
  const int64_t po = T.piv_off[t];
  const double* Dd = S.Dd + po;
  const double* De = S.De + po;
  const int8_t* pv = S.piv + po;
  for (int32_t c = threadIdx.x; c < r; c += blockDim.x) {
    su[c] = balance_shift(Dd, De, pv, c0 + c);
    const int8_t pt = pv[c0 + c];
    wpt[c] = pt;
    wself[c] = Dd[c0 + c];
    woth[c] = pt == 1 ? 0.0 : (pt == 2 ? De[c0 + c] : De[c0 + c - 1]);
  }
  __syncthreads();
  const int32_t nq = (r + 15) / 16 * 2;          // 8-column blocks covering the padded window
  const int NG = nq >= 8 ? 8 : (nq >= 4 ? 4 : 2);
  const int RT = kSThreads / NG;                 // rows per pass
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int64_t rows = m - s;
  const int lr = threadIdx.x % RT, g = threadIdx.x / RT;
  for (int64_t rb = static_cast<int64_t>(blockIdx.x) * RT; rb < rows; rb += static_cast<int64_t>(gridDim.x) * RT) {
    const int64_t row = rb + lr;
    const bool ok = row < rows;
    int ex = kNoExp, ey = kNoExp;
    if (ok)
      for (int32_t q = g; q < nq; q += NG)
        for (int32_t c = q * 8; c < min(q * 8 + 8, r); ++c) {
          const int u = su[c];
          const int bx = bexp(L[static_cast<int64_t>(c0 + c) * ld + s + row]);
          const int by = row < wrows ? bexp(wval_s(L, ld, s + row, c0 + c, c, wself, woth, wpt)) : 0;
          if (bx) ex = max(ex, bx - u);
          if (by) ey = max(ey, by + u);
        }
    smx[0][threadIdx.x] = ex;
    smx[1][threadIdx.x] = ey;
    __syncthreads();
    int mx = kNoExp, my = kNoExp;
    for (int q = 0; q < NG; ++q) {
      mx = max(mx, smx[0][q * RT + lr]);
      my = max(my, smx[1][q * RT + lr]);
    }
    __syncthreads();
    const int el = mx != kNoExp ? mx - 1021 : 0;   // |x 2^-u| < 2^{el-1} along the row
    const int ew = my != kNoExp ? my - 1021 : 0;
    if (!ok) continue;
    if (g == 0) { E.eL[row] = el; E.eW[row] = ew; }
    for (int32_t q = g; q < nq; q += NG) {
#pragma unroll 1
      for (int which = 0; which < (row < wrows ? 2 : 1); ++which) {
        uint32_t pk[ND][4];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int32_t c = q * 8 + e;
          double x = 0.0;
          int u = 0;
          if (c < r) {
            u = su[c];
            x = which == 0 ? L[static_cast<int64_t>(c0 + c) * ld + s + row]
                           : wval_s(L, ld, s + row, c0 + c, c, wself, woth, wpt);
          }
          uint32_t d[ND];
          balanced_digits<ND>(x, which == 0 ? u : -u, which == 0 ? el : ew, d);
#pragma unroll
          for (int a = 0; a < ND; ++a) {
            if (e % 2 == 0) pk[a][e / 2] = d[a];
            else pk[a][e / 2] |= d[a] << 16;
          }
        }
#pragma unroll
        for (int a = 0; a < ND; ++a)
          *reinterpret_cast<uint4*>(which == 0 ? E.Ls + ldig_off<ND>(a, q, row) : E.Ws + wdig_off<ND>(a, q, row)) =
              make_uint4(pk[a][0], pk[a][1], pk[a][2], pk[a][3]);
      }
    }
  }
}

// Tiles of the lower triangle of [s, m): i-blocks of 128 rows, j-blocks of 32.  Bands of kBand
// i-blocks are taken in turn; inside a band the order is j-major, so the concurrently running
// tiles share their j-blocks (the W digits are read from memory about once per band).  Slots of
// a band's rectangle above the diagonal or past the last j-block are empty (false).
constexpr int kBand = 8;
KEP_D int64_t tile_slots(int64_t nI, int64_t nJ) {
  int64_t n = 0;
  for (int64_t I0 = 0; I0 < nI; I0 += kBand) {
    const int64_t I1 = min(I0 + kBand, nI);
    n += (I1 - I0) * min(4 * I1, nJ);
  }
  return n;
}
// Slot t -> tile (I, J) in closed form (32-bit): the first bands are 8 high and 32 (b + 1) wide
// (prefix 128 b (b + 1)), the following 8-high bands are nJ wide, and a last band may be lower.
KEP_D bool tile_ij(int t, int nI, int nJ, int& I, int& J) {
  const int nfull = min(nI / 8, nJ / 32);
  const int pf = 128 * nfull * (nfull + 1);
  if (t < pf) {
    int b = static_cast<int>((sqrtf(1.0f + static_cast<float>(t) / 32.0f) - 1.0f) * 0.5f);
    while (b > 0 && 128 * b * (b + 1) > t) --b;
    while (128 * (b + 1) * (b + 2) <= t) ++b;
    const int r = t - 128 * b * (b + 1);
    J = r >> 3;
    I = 8 * b + (r & 7);
    return J < 4 * (I + 1);
  }
  t -= pf;
  int I0 = 8 * nfull;
  if (32 * (nfull + 1) > nJ) {
    const int nb2 = (nI - I0) / 8;
    if (t < nb2 * 8 * nJ) {
      const int bb = t / (8 * nJ), rr = t - bb * 8 * nJ;
      J = rr >> 3;
      I = I0 + 8 * bb + (rr & 7);
      return J < 4 * (I + 1);
    }
    t -= nb2 * 8 * nJ;
    I0 += 8 * nb2;
  }
  if (I0 >= nI) return false;
  const int h = nI - I0, w = min(4 * nI, nJ);
  if (t >= h * w) return false;
  J = t / h;
  I = I0 + t % h;
  return J < 4 * (I + 1);
}

// C - (hi 2^32 + lo) 2^scale for |hi|, |lo| < 2^52.  The integer V = hi 2^32 + lo is brought to
// 64 bits as V = +-(T + f) 2^sh with an integer T < 2^56 and 0 <= f < 1; T and a sticky bit for
// f != 0 then go through one correctly rounded int64 -> double conversion (2T + sticky has at
// least 55 significant bits whenever f can be nonzero, so the sticky bit only breaks ties, which
// rounds V to nearest), the power of two enters the exponent field, and one FP64 subtraction
// follows.  Scaled values below 2^-1000 are treated as zero.
KEP_D double sub_scaled(double C, long long hi, long long lo, int scale) {
  const unsigned long long ah = static_cast<unsigned long long>(hi < 0 ? -hi : hi);
  const int sh = max(0, 41 - __clzll(static_cast<long long>(ah)));   // bit length of |hi| minus 23
  long long T2;                                  // 2T + sticky, with the sign of V
  if (sh == 0) {                                 // |hi| < 2^23: V is exact in 64 bits, |V| < 2^56
    T2 = (static_cast<long long>(static_cast<unsigned long long>(hi) << 32) + lo) * 2;
  } else {                                       // V has the sign of hi
    const long long h2 = hi < 0 ? -hi : hi, l2 = hi < 0 ? -lo : lo;
    const long long T = (h2 << (32 - sh)) + (l2 >> sh);
    const long long st = (static_cast<unsigned long long>(l2) & ((1ull << sh) - 1)) != 0ull ? 1 : 0;
    T2 = hi < 0 ? -(2 * T + st) : 2 * T + st;
  }
  const double d = __ll2double_rn(T2);           // V 2^{1-sh}, rounded once
  const int e = sh - 1 + scale;                  // d 2^e = V 2^scale
  const long long db = __double_as_longlong(d);
  const int ed = static_cast<int>((db >> 52) & 0x7ff);
  if (ed == 0 || ed + e < 24) return C;          // zero, or below 2^-1000
  if (ed + e > 2046) return C - copysign(__longlong_as_double(0x7ff0000000000000ll), d);
  return C - __longlong_as_double(db + (static_cast<long long>(e) << 52));
}

// Exact integer from an FP32 level sum that holds an integer (|v| <= 2^24).
KEP_D int level_int(float v) { return __float2int_rn(v); }

// The level sums of one entry over one half window (x[g]: level g+2, |x[g]| <= 2^24) added in
// base 256 to levels 2..5 (vh) and 6..9 (vl).  Fast path: with every level sum at most 2^22 in
// magnitude, v + 1.5 2^23 lands in [2^23, 2^24], where the float's bits minus those of 1.5 2^23
// are the integer v (the constant offsets are taken out in one step); otherwise (rare) each sum
// is converted on its own.
constexpr float kMagic = 12582912.0f;          // 1.5 2^23
constexpr int kMagicBits = 0x4B400000;
KEP_D void add_levels(const float (&x)[8], long long& vh, long long& vl) {
  float big = 0.f;
#pragma unroll
  for (int g = 0; g < 8; ++g) big = fmaxf(big, fabsf(x[g]));
  if (big <= 4194304.0f) {
    unsigned b[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) b[g] = __float_as_uint(x[g] + kMagic);
    // (b0 - K) 256 + (b1 - K) = b0 256 + b1 - 257 K: exact modulo 2^32, and the result fits
    constexpr unsigned kOff = 257u * static_cast<unsigned>(kMagicBits);
    const int p0 = static_cast<int>(b[0] * 256u + b[1] - kOff), p1 = static_cast<int>(b[2] * 256u + b[3] - kOff);
    const int p2 = static_cast<int>(b[4] * 256u + b[5] - kOff), p3 = static_cast<int>(b[6] * 256u + b[7] - kOff);
    vh += static_cast<long long>(p0) * 65536 + p1;
    vl += static_cast<long long>(p2) * 65536 + p3;
  } else {
    int l[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) l[g] = level_int(x[g]);
    vh += (static_cast<long long>(l[0]) << 24) + (static_cast<long long>(l[1]) << 16) +
          (static_cast<long long>(l[2]) << 8) + l[3];
    vl += (static_cast<long long>(l[4]) << 24) + (static_cast<long long>(l[5]) << 16) +
          (static_cast<long long>(l[6]) << 8) + l[7];
  }
}

constexpr int kMaxBatch = 512;              // fronts per tensor-core launch

template <bool kWin, int S>
__global__ void __launch_bounds__(kFlushThreads, 1) lf_flush_tc_kernel(FrontTables T, SlotSet SS,
                                                                       LargeWork W, EmulBatch BA,
                                                                       unsigned long long* flops) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  // per entry of the batch: tile-slot prefix, tile grid, 16-column steps, first row, end column
  __shared__ int pre[kMaxBatch + 1];
  __shared__ int enI[kMaxBatch], enJ[kMaxBatch], eKS[kMaxBatch], eS[kMaxBatch], eCE[kMaxBatch];
  for (int e = threadIdx.x; e < BA.nb; e += blockDim.x) {
    const int32_t b = BA.e0 + e, t = BA.lf[b];
    const int32_t m = T.m_sym[t] + SS.s[emul_shift(BA, b)].d_in[t];
    int32_t c0, c1, s, ce;
    int nI = 0, nJ = 0, KS = 0, ns = 0;
    if (emul_range<kWin>(W, b, m, c0, c1, s, ce)) {
      const int32_t r = c1 - c0;
      KS = (r + 15) / 16;
      const int64_t h = m - s, w = ce - s;
      nI = static_cast<int>((h + kTM - 1) / kTM);
      nJ = static_cast<int>((w + kTN - 1) / kTN);
      ns = static_cast<int>(tile_slots(nI, nJ));
      if (blockIdx.x == 0) {
        // tensor-core work issued (i-block I has min(4I + 4, nJ) tiles), and the FP64 update it
        // stands for (2 r per updated entry)
        const int64_t c = min(nI, nJ / 4);
        const int64_t ntiles = 2 * c * (c + 1) + (nI - c) * static_cast<int64_t>(nJ);
        atomicAdd(&flops[KC_FLUSH_TC],
                  static_cast<unsigned long long>(2ll * kTM * (S * (S + 1) / 2) * kTN * 16 * KS * ntiles));
        atomicAdd(&flops[KC_COUNT], static_cast<unsigned long long>(2 * static_cast<int64_t>(r) * (w * h - w * (w - 1) / 2)));
      }
      eS[e] = s;
      eCE[e] = ce;
    }
    enI[e] = nI; enJ[e] = nJ; eKS[e] = KS; pre[e + 1] = ns;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    pre[0] = 0;
    for (int e = 0; e < BA.nb; ++e) pre[e + 1] += pre[e];
  }
  __syncthreads();
  const int nslots = pre[BA.nb];
  if (static_cast<int>(blockIdx.x) >= nslots) return;
  // slot -> (entry, tile): the entry is the last one whose prefix is <= slot (a nonempty one)
  auto locate = [&](int slot, int& e, int& I, int& J) -> bool {
    int lo = 0, hi = BA.nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (pre[mid] <= slot) lo = mid; else hi = mid - 1;
    }
    e = lo;
    return tile_ij(slot - pre[e], enI[e], enJ[e], I, J);
  };
  unsigned char* sbase =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) { tc::mbar_init(&full_bar[i], 1); tc::mbar_init(&empty_bar[i], 1); }
    for (int i = 0; i < 2; ++i) { tc::mbar_init(&tfull_bar[i], 1); tc::mbar_init(&tempty_bar[i], kEpiWarps * 32); }
    tc::mbar_init(&drain_bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, Split<S>::kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  if (warp == kEpiWarps) {
    // ---- producer: one bulk copy per operand per 16-column step ----
    if (lane == 0) {
      int64_t f = 0;
      bool ok = true;
      for (int slot = blockIdx.x; slot < nslots && ok; slot += gridDim.x) {
        int e, I, J;
        if (!locate(slot, e, I, J)) continue;
        const EmulArgs E = entry_args(BA, e, T.m_alloc[BA.lf[BA.e0 + e]]);
        const int KS = eKS[e];
        for (int kk = 0; kk < KS; ++kk, ++f) {
          const int st = static_cast<int>(f % kStages);
          if (f >= kStages &&
              !tc::mbar_wait(&empty_bar[st], static_cast<uint32_t>((f / kStages - 1) & 1), kWaitNs, kSleepCopy)) {
            ok = false;
            break;
          }
          unsigned char* sa = sbase + static_cast<size_t>(st) * Split<S>::kStageBytes;
          tc::mbar_arrive_expect_tx(&full_bar[st], Split<S>::kStageBytes);
          tc::bulk_g2s(sa, E.Ls + ldig_off<S>(0, 2 * kk, I * kTM), Split<S>::kStageA, &full_bar[st]);
          tc::bulk_g2s(sa + Split<S>::kStageA, E.Ws + wdig_off<S>(0, 2 * kk, J * kTN), Split<S>::kStageB,
                       &full_bar[st]);
        }
      }
      if (!ok) {
        abort_flag = 1;
        // let the copies already issued land before the CTA can exit
        for (int64_t g = f - 1; g >= 0 && g >= f - kStages; --g)
          tc::mbar_wait(&full_bar[g % kStages], static_cast<uint32_t>((g / kStages) & 1), kWaitNs);
      }
    }
  } else if (warp == kEpiWarps + 1) {
    // ---- MMA issue: per step, slice a of L against the stacked slices 1 .. 8-a of W ----
    if (lane == 0) {
      const uint32_t s0 = tc::smem_addr(sbase);
      int64_t f = 0, u = 0;                     // steps, half-window accumulations issued
      bool ok = true;
      for (int slot = blockIdx.x; slot < nslots && ok; slot += gridDim.x) {
        int e, I, J;
        if (!locate(slot, e, I, J)) continue;
        const int KS = eKS[e], NH = (KS + kHalf - 1) / kHalf;
        for (int hh = 0; hh < NH && ok; ++hh, ++u) {
          const int buf = static_cast<int>(u & 1);
          if (u >= 2 && !tc::mbar_wait(&tempty_bar[buf], static_cast<uint32_t>(((u >> 1) - 1) & 1), kWaitNs, kSleepMma)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t dbase = tmem + static_cast<uint32_t>(buf * S * kTN);
          const int k1 = min(KS, (hh + 1) * kHalf);
          for (int kk = hh * kHalf; kk < k1; ++kk, ++f) {
            const int st = static_cast<int>(f % kStages);
            if (!tc::mbar_wait(&full_bar[st], static_cast<uint32_t>((f / kStages) & 1), kWaitNs, kSleepMma)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t sa = s0 + st * Split<S>::kStageBytes, sb = sa + Split<S>::kStageA;
            const uint64_t bdesc = tc::smem_desc(sb, Split<S>::kStageB / 2, 128);
            const uint64_t adesc = tc::smem_desc(sa, Split<S>::kStageA / 2, 128);
#pragma unroll
            for (int a = 0; a < S; ++a)   // levels a+2 .. S+1 at columns 32 a ..; slice a of L
              tc::mma_bf16(dbase + static_cast<uint32_t>(a * kTN), adesc + static_cast<uint64_t>(a * (kTM * 16 / 16)),
                           bdesc, tc::idesc_bf16(kTM, (S - a) * kTN),
                           (kk > hh * kHalf || a > 0) ? 1u : 0u);
            tc::mma_commit(&empty_bar[st]);
          }
          if (!ok) break;
          tc::mma_commit(&tfull_bar[buf]);
        }
      }
      if (!ok) abort_flag = 1;
      tc::mma_commit(&drain_bar);               // all MMAs of this CTA done before tensor memory goes
      tc::mbar_wait(&drain_bar, 0, kWaitNs);
    }
  } else {
    // ---- epilogue: warp w reads lanes (rows) 32 (w % 4) .. +31, columns 8 (w / 4) .. +7 ----
    constexpr int kCols = kTN / (kEpiWarps / 4);
    const int quarter = warp & 3, c_lo = (warp >> 2) * kCols;
    const uint32_t trow = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
    int64_t u = 0;
    bool ok = true;
    for (int slot = blockIdx.x; slot < nslots && ok; slot += gridDim.x) {
      int e, I, J;
      if (!locate(slot, e, I, J)) continue;
      const int32_t t = BA.lf[BA.e0 + e];
      const int32_t g = emul_shift(BA, BA.e0 + e);
      const FrontView v = front_view(T, SS.s[g], SS.cbpool[g], t, SS.s[g].d_in[t]);
      const EmulArgs E = entry_args(BA, e, T.m_alloc[t]);
      const int32_t s = eS[e], ce = eCE[e];
      const int NH = (eKS[e] + kHalf - 1) / kHalf;
      // this thread's row and its entries of C (column stride cs from the entry of column j0; the
      // columns of a tile lie on one side of p except at one j-block of the front); they are
      // brought into L2 while the MMAs run
      const int64_t i = s + static_cast<int64_t>(I) * kTM + quarter * 32 + lane;
      const int64_t j0 = s + static_cast<int64_t>(J) * kTN + c_lo;
      const bool rowok = i < v.m && j0 <= i;
      const bool split = j0 < v.p && j0 + kCols > v.p;
      double* cp = rowok ? v.at(static_cast<int32_t>(i), static_cast<int32_t>(j0)) : nullptr;
      const int64_t cs = j0 < v.p ? v.ldL : v.c;
      auto centry = [&](int c) {
        return split ? v.at(static_cast<int32_t>(i), static_cast<int32_t>(j0 + c)) : cp + c * cs;
      };
      if (rowok)
#pragma unroll
        for (int c = 0; c < kCols; ++c)
          if (j0 + c <= i && j0 + c < ce) asm volatile("prefetch.global.L2 [%0];" ::"l"(centry(c)));
      long long vh[kCols], vl[kCols];
#pragma unroll
      for (int c = 0; c < kCols; ++c) { vh[c] = 0; vl[c] = 0; }
      for (int hh = 0; hh < NH; ++hh, ++u) {
        const int buf = static_cast<int>(u & 1);
        if (!tc::mbar_wait(&tfull_bar[buf], static_cast<uint32_t>((u >> 1) & 1), kWaitNs, kSleepEpi)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t tb = trow + static_cast<uint32_t>(buf * S * kTN);
#pragma unroll
        for (int cg = 0; cg < kCols / 4; ++cg) {
          uint32_t x[S][4];
#pragma unroll
          for (int g = 0; g < S; ++g) tc::tmem_ld4(tb + g * kTN + c_lo + cg * 4, x[g]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int g = 0; g < S; ++g) tc::tmem_keep(x[g]);
#pragma unroll
          for (int ee = 0; ee < 4; ++ee) {
            float xs[S];
#pragma unroll
            for (int g = 0; g < S; ++g) xs[g] = __uint_as_float(x[g][ee]);
            if constexpr (S == kSlices) {
              add_levels(xs, vh[cg * 4 + ee], vl[cg * 4 + ee]);
            } else {
              // levels 2 .. S+1 in base 256 (each sum an exact integer of at most 2^23)
              long long v = 0;
#pragma unroll
              for (int g = 0; g < S; ++g) v = v * 256 + level_int(xs[g]);
              vl[cg * 4 + ee] += v;
            }
          }
        }
        // this buffer is free for the MMAs of a later half window
        tc::fence_before_sync();
        tc::mbar_arrive(&tempty_bar[buf]);
      }
      if (!ok) {
        abort_flag = 1;
        break;
      }
      if (rowok) {
        const int ei = E.eL[i - s] - Split<S>::kShift;
        // all loads first (the stores below could alias them as far as the compiler knows)
        double cv[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) cv[c] = (j0 + c <= i && j0 + c < ce) ? *centry(c) : 0.0;
#pragma unroll
        for (int c = 0; c < kCols; ++c)
          if (j0 + c <= i && j0 + c < ce) *centry(c) = sub_scaled(cv[c], vh[c], vl[c], ei + E.eW[j0 + c - s]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag)
    for (int g = 0; g < SS.n; ++g) atomicOr(&SS.s[g].status[0], ST_TIMEOUT);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, Split<S>::kTmemCols);
  }
}

}  // namespace

void emul_init() {
  // once per process (a function-local static is initialised once even when contexts on several
  // host threads get here together); called before any stream capture
  static const bool attr_set = [] {
    cudaFuncSetAttribute(lf_flush_tc_kernel<true, kSlices>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(Split<kSlices>::kSmem));
    cudaFuncSetAttribute(lf_flush_tc_kernel<false, kSlices>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(Split<kSlices>::kSmem));
    cudaFuncSetAttribute(lf_flush_tc_kernel<true, kSlicesLow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(Split<kSlicesLow>::kSmem));
    cudaFuncSetAttribute(lf_flush_tc_kernel<false, kSlicesLow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(Split<kSlicesLow>::kSmem));
    return true;
  }();
  (void)attr_set;
}

size_t emul_workspace_bytes(int64_t cap_rows) {
  const int64_t R = digit_pitch(cap_rows);
  return 2ull * kSlices * kKB * R * 8 * sizeof(__nv_bfloat16) + 2ull * R * sizeof(int32_t) + 512;
}

// Window update (window = true) or flush for the batch entries e0 .. e0 + nb - 1 (fronts on the
// tensor-core path; entry e's workspace at ws + d_off[e]); the kernels skip entries without that
// update this step.
void launch_emul_update(bool window, bool low, const FrontTables& T, const SlotSet& SS, const LargeWork& W,
                        const Batch& B, int32_t nb, void* ws, const int64_t* d_off, int64_t rows_hint,
                        cudaStream_t st, int num_sms, Timer* timer, unsigned long long* flops) {
  emul_init();
  EmulBatch BA;
  BA.ws = static_cast<unsigned char*>(ws);
  BA.off = d_off;
  BA.lf = B.lf;
  BA.sh = B.sh;
  BA.e0 = B.e0;
  BA.nb = nb;
  const int gs = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows_hint + 31) / 32,
                                                                          std::max(1, num_sms * 8 / nb))));
  auto go = [&](auto win, auto nd) {
    constexpr bool W_ = decltype(win)::value;
    constexpr int S_ = decltype(nd)::value;
    KEP_LAUNCH(timer, KC_SLICE, st, (lf_slice_kernel<W_, S_><<<dim3(gs, nb), kSThreads, 0, st>>>(T, SS, W, BA)));
    KEP_LAUNCH(timer, KC_FLUSH_TC, st,
               (lf_flush_tc_kernel<W_, S_><<<num_sms, kFlushThreads, Split<S_>::kSmem, st>>>(T, SS, W, BA, flops)));
  };
  using T8 = std::integral_constant<int, kSlices>;
  using TL = std::integral_constant<int, kSlicesLow>;
  if (window) {
    if (low) go(std::true_type{}, TL{}); else go(std::true_type{}, T8{});
  } else {
    if (low) go(std::false_type{}, TL{}); else go(std::false_type{}, T8{});
  }
}

int32_t emul_max_batch() { return kMaxBatch; }

}  // namespace kep
