// FP64-accurate Schur update on the tensor cores (the window flush of the front factorization).
//
// C(i, j) -= sum_c L(i, c) W(j, c), W = L D, for the pivots of one window (rank r <= 256).  GB300
// issues FP64 FMAs at about 1/64 of its FP32 rate, so the product is formed from bf16 pieces
// whose products the tensor cores sum exactly (an error-free splitting in the manner of Ozaki et
// al.):
//
//  * column balancing: column c of L is scaled by 2^{-u_c} and column c of W by 2^{u_c} (u_c from
//    the two columns' largest exponents), which leaves every product unchanged and keeps the
//    spread of D out of the rows;
//  * every row is scaled by a power of two 2^e with |x| < 2^{e-1} for all its entries, and
//    |x| 2^{8-e} (< 128) is written in balanced base-256 digits, sum_a d_a 256^{1-a}, a = 1..8,
//    d_1 in [0, 128], d_a in [-128, 127] otherwise, cut from the double's significand with integer
//    operations (the dropped tail is below 2^-63 of 2^e); each digit times the sign of x is exact
//    in bf16 and every digit product is at most 2^14 in magnitude;
//  * the tensor cores (tcgen05, accumulators in tensor memory) sum, for each level g = a + b
//    (2 <= g <= 9), the products s_a(i, c) t_b(j, c) over the whole window in two FP32
//    accumulators, one for a <= 4 and one for a >= 5.  Each holds at most 4 pairs x 256 columns x
//    2^14 = 2^24 in magnitude, integers all along, so every FP32 sum is exact;
//  * the twelve exact level sums of an entry are combined in integers and C(i, j) receives
//    -2^{e_i + f_j - 72} (V_hi 2^32 + V_lo), rounded once to FP64.
//
// The only roundings are the one FP64 product L D, the dropped digit tail and the final FP64
// conversion and subtraction: as accurate as an FP64 rank-r update.
//
// Tensor-core layout: a CTA owns a 128 x 32 tile of C (rows i, columns j).  Per 16-column step it
// issues eight MMAs, slice a of the L rows (M = 128) against slices 1 .. 9-a of the W rows stacked
// along N (N = 32 (9-a)), writing the accumulators of levels a+1 .. 9 side by side in tensor
// memory; both operands are staged in shared memory by bulk copies in a five-step pipeline.
#include <algorithm>

#include <cuda_bf16.h>

#include "kep_tc.cuh"

namespace kep {

namespace {

constexpr int kSlices = 8;
constexpr int kKB = kWindow / 8;              // 8-column blocks of a window
constexpr int kTM = 128;                      // tile rows (i): tensor-memory lanes
constexpr int kTN = 32;                       // tile columns (j) per digit of W
constexpr int kStages = 5;                    // shared-memory pipeline depth (16 columns each)
constexpr uint32_t kStageA = 2 * kSlices * kTM * 16;   // [k-block 2][slice 8][row 128][16 B]
constexpr uint32_t kStageB = 2 * kSlices * kTN * 16;   // [k-block 2][slice 8][row 32][16 B]
constexpr uint32_t kStageBytes = kStageA + kStageB;
constexpr size_t kFlushSmem = static_cast<size_t>(kStages) * kStageBytes + 1024;
constexpr int kFlushThreads = 192;            // warps 0-3 epilogue, 4 copies, 5 MMA issue
constexpr uint32_t kTmemCols = 512;           // 8 + 4 level accumulators x 32 columns (384 used)
constexpr uint64_t kWaitNs = 2000000000ull;   // bounded waits: 2 s
constexpr int kNoExp = -(1 << 20);            // row maximum of an all-zero row

struct EmulArgs {
  __nv_bfloat16* Ls;   // digits of the balanced, scaled L rows: [slice][k-block][row (pitch R)][8]
  __nv_bfloat16* Ws;   // same for W
  double* Wv;          // [kWindow][cap_rows] W = L D (column-major, like L)
  int32_t* eL;         // [R] row scale exponents
  int32_t* eW;
  int32_t* cexp;       // [2][kWindow] largest biased exponent of |L(., c)| and |W(., c)|
  int64_t cap_rows;
  int64_t R;           // row pitch of the digit arrays (>= rows + kTM)
};

KEP_HD int64_t digit_pitch(int64_t cap_rows) { return (cap_rows + kTM - 1) / kTM * kTM + kTM; }

KEP_D int bexp(double x) {                    // biased exponent field (0 for zero / subnormal)
  return static_cast<int>((__double_as_longlong(x) >> 52) & 0x7ff);
}

// W(i, c) = sum_c' L(i, c') D(c', c) for the window's pivot c (2x2 blocks mix two columns)
KEP_D double wval(const double* L, int64_t ld, int64_t i, int32_t c, const double* Dd, const double* De,
                  const int8_t* pv) {
  const double x = L[static_cast<int64_t>(c) * ld + i];
  const int8_t pt = pv[c];
  if (pt == 1) return x * Dd[c];
  if (pt == 2) return x * Dd[c] + L[static_cast<int64_t>(c + 1) * ld + i] * De[c];
  return L[static_cast<int64_t>(c - 1) * ld + i] * De[c - 1] + x * Dd[c];
}

KEP_D int balance_shift(const EmulArgs& E, int32_t c) {
  const int ex = E.cexp[c], ey = E.cexp[kWindow + c];
  if (ex == 0 || ey == 0) return 0;
  const int d = ex - ey;
  return d >= 0 ? d / 2 : -((-d + 1) / 2);     // floor(d / 2)
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

// bf16 bit pattern of the integer d, |d| <= 128 (exact: at most 8 significant bits)
KEP_D uint32_t digit_bits(int d) { return __float_as_uint(__int2float_rn(d)) >> 16; }

// The eight balanced digits of one value, times its sign, as bf16 bit patterns.
KEP_D void balanced_digits(double x, int u, int e, uint32_t (&d)[kSlices]) {
  const unsigned long long Y = fixed64(x, u, e) + 0x0080808080808080ull;   // pre-carry of the low 7
  const bool neg = x < 0.0;
#pragma unroll
  for (int a = 0; a < kSlices; ++a) {
    const int v = a == 0 ? static_cast<int>(Y >> 56) : static_cast<int>((Y >> (56 - 8 * a)) & 0xff) - 128;
    d[a] = digit_bits(neg ? -v : v);
  }
}

// Pass 1: W = L D for the window's columns over the rows [we, m), and per column the largest
// exponents of |L| and |W| (CTAs over row chunks, one thread per column).
__global__ void __launch_bounds__(256) lf_colmax_kernel(FrontTables T, FactorSlot S, LargeWork W, const int32_t* lf,
                                                        int32_t b, EmulArgs E) {
  if (W.done[b] || !W.flush[b]) return;
  const int32_t t = lf[b];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t c0 = W.ws[b], c1 = W.kend[b], s = W.we[b];
  const int32_t r = c1 - c0;
  if (r <= 0 || s >= m) return;
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int64_t po = T.piv_off[t];
  const int64_t rows = m - s;
  // threads over rows (coalesced), loop over the window's columns
  const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  __shared__ int sx[kWindow], sy[kWindow];
  for (int32_t c = threadIdx.x; c < kWindow; c += blockDim.x) { sx[c] = 0; sy[c] = 0; }
  __syncthreads();
  for (int32_t c = 0; c < r; ++c) {
    int mx = 0, my = 0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
      const int64_t i = s + row;
      const double x = L[static_cast<int64_t>(c0 + c) * ld + i];
      const double y = wval(L, ld, i, c0 + c, S.Dd + po, S.De + po, S.piv + po);
      E.Wv[static_cast<int64_t>(c) * E.cap_rows + row] = y;
      mx = max(mx, bexp(x));
      my = max(my, bexp(y));
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      my = max(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) { atomicMax(&sx[c], mx); atomicMax(&sy[c], my); }
  }
  __syncthreads();
  for (int32_t c = threadIdx.x; c < r; c += blockDim.x) {
    atomicMax(&E.cexp[c], sx[c]);
    atomicMax(&E.cexp[kWindow + c], sy[c]);
  }
}

// Pass 2: per row, the scale exponents of the balanced L and W rows, then the digits of every
// entry of the window (zero up to the next multiple of 16 columns).  Thread (row, half): the
// half's 8-column blocks; each 16-byte store holds one row's 8 digits of one slice and block,
// consecutive threads writing consecutive rows.
constexpr int kSRows = 128;
__global__ void __launch_bounds__(256) lf_slice_kernel(FrontTables T, FactorSlot S, LargeWork W, const int32_t* lf,
                                                       int32_t b, EmulArgs E) {
  __shared__ int smx[2][2][kSRows];
  if (W.done[b] || !W.flush[b]) return;
  const int32_t t = lf[b];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t c0 = W.ws[b], c1 = W.kend[b], s = W.we[b];
  const int32_t r = c1 - c0;
  if (r <= 0 || s >= m) return;
  const int32_t nq = (r + 15) / 16 * 2;          // 8-column blocks covering the padded window
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int64_t rows = m - s;
  const int lr = threadIdx.x % kSRows, half = threadIdx.x / kSRows;
  for (int64_t rb = static_cast<int64_t>(blockIdx.x) * kSRows; rb < rows; rb += static_cast<int64_t>(gridDim.x) * kSRows) {
    const int64_t row = rb + lr;
    const bool ok = row < rows;
    int ex = kNoExp, ey = kNoExp;
    if (ok)
      for (int32_t c = half; c < r; c += 2) {
        const int u = balance_shift(E, c);
        const int bx = bexp(L[static_cast<int64_t>(c0 + c) * ld + s + row]);
        const int by = bexp(E.Wv[static_cast<int64_t>(c) * E.cap_rows + row]);
        if (bx) ex = max(ex, bx - u);
        if (by) ey = max(ey, by + u);
      }
    smx[0][half][lr] = ex;
    smx[1][half][lr] = ey;
    __syncthreads();
    const int mx = max(smx[0][0][lr], smx[0][1][lr]), my = max(smx[1][0][lr], smx[1][1][lr]);
    __syncthreads();
    const int el = mx != kNoExp ? mx - 1021 : 0;   // |x 2^-u| < 2^{el-1} along the row
    const int ew = my != kNoExp ? my - 1021 : 0;
    if (!ok) continue;
    if (half == 0) { E.eL[row] = el; E.eW[row] = ew; }
    for (int32_t q = half; q < nq; q += 2) {
#pragma unroll 1
      for (int which = 0; which < 2; ++which) {
        uint32_t pk[kSlices][4];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int32_t c = q * 8 + e;
          double x = 0.0;
          int u = 0;
          if (c < r) {
            u = balance_shift(E, c);
            x = which == 0 ? L[static_cast<int64_t>(c0 + c) * ld + s + row]
                           : E.Wv[static_cast<int64_t>(c) * E.cap_rows + row];
          }
          uint32_t d[kSlices];
          balanced_digits(x, which == 0 ? u : -u, which == 0 ? el : ew, d);
#pragma unroll
          for (int a = 0; a < kSlices; ++a) {
            if (e % 2 == 0) pk[a][e / 2] = d[a];
            else pk[a][e / 2] |= d[a] << 16;
          }
        }
        __nv_bfloat16* base = which == 0 ? E.Ls : E.Ws;
#pragma unroll
        for (int a = 0; a < kSlices; ++a)
          *reinterpret_cast<uint4*>(base + ((static_cast<int64_t>(a) * kKB + q) * E.R + row) * 8) =
              make_uint4(pk[a][0], pk[a][1], pk[a][2], pk[a][3]);
      }
    }
  }
}

// Tiles of the lower triangle of [s, m): i-blocks of 128 rows, j-blocks of 32; i-block I pairs
// with j-blocks 0 .. 4I+3 (the last one with all j-blocks).
KEP_D void tile_ij(int64_t t, int64_t nI, int64_t& I, int64_t& J) {
  const int64_t full = 2 * (nI - 1) * nI;
  if (t >= full) { I = nI - 1; J = t - full; return; }
  int64_t i = static_cast<int64_t>((sqrt(1.0 + 2.0 * static_cast<double>(t)) - 1.0) * 0.5);
  while (i > 0 && 2 * i * (i + 1) > t) --i;
  while (2 * (i + 1) * (i + 2) <= t) ++i;
  I = i;
  J = t - 2 * i * (i + 1);
}

// (hi 2^32 + lo) 2^scale rounded to the nearest double (ties to even), integer operations only;
// |hi|, |lo| < 2^62.  Results below the normal range are flushed to zero.
KEP_D double combine_to_double(long long hi, long long lo, int scale) {
  unsigned long long L = (static_cast<unsigned long long>(hi) << 32) + static_cast<unsigned long long>(lo);
  const unsigned long long carry = L < (static_cast<unsigned long long>(hi) << 32) ? 1ull : 0ull;
  const long long H = (hi >> 32) + (lo >> 63) + static_cast<long long>(carry);
  const bool neg = H < 0;
  unsigned long long uh = static_cast<unsigned long long>(H);
  if (neg) {
    L = ~L + 1ull;
    uh = ~uh + (L == 0ull ? 1ull : 0ull);
  }
  int lz;
  unsigned long long top, rest;
  if (uh != 0ull) {
    lz = __clzll(static_cast<long long>(uh));
    top = lz ? (uh << lz) | (L >> (64 - lz)) : uh;
    rest = L << lz;
  } else {
    if (L == 0ull) return 0.0;
    lz = 64 + __clzll(static_cast<long long>(L));
    top = L << (lz - 64);
    rest = 0ull;
  }
  unsigned long long mant = top >> 11;          // 53 bits, leading one at bit 52
  const unsigned long long rbit = (top >> 10) & 1ull;
  const bool sticky = (top & 0x3ffull) != 0ull || rest != 0ull;
  mant += rbit & ((sticky ? 1ull : 0ull) | (mant & 1ull));
  const int E = 127 - lz + scale + 1023;        // biased exponent of the leading bit
  if (E <= 0) return 0.0;
  const unsigned long long bits = (static_cast<unsigned long long>(E - 1) << 52) + mant;
  return __longlong_as_double(static_cast<long long>(bits | (neg ? (1ull << 63) : 0ull)));
}

// Exact integer from an FP32 level sum that holds an integer (|v| <= 2^24).
KEP_D int level_int(uint32_t bits) { return __float2int_rn(__uint_as_float(bits)); }

__global__ void __launch_bounds__(kFlushThreads, 1) lf_flush_tc_kernel(FrontTables T, FactorSlot S, double* cbpool,
                                                                       LargeWork W, const int32_t* lf, int32_t b,
                                                                       EmulArgs E, unsigned long long* flops) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t tfull_bar, tempty_bar, drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  if (W.done[b] || !W.flush[b]) return;
  if (blockIdx.x == 0)                        // column exponents are used up: clear for the next window
    for (int32_t c = threadIdx.x; c < 2 * kWindow; c += blockDim.x) E.cexp[c] = 0;
  const int32_t t = lf[b];
  const int32_t d_in = S.d_in[t];
  const FrontView v = front_view(T, S, cbpool, t, d_in);
  const int32_t c0 = W.ws[b], c1 = W.kend[b], s = W.we[b];
  const int32_t r = c1 - c0;
  if (r <= 0 || s >= v.m) return;
  const int KS = (r + 15) / 16;               // 16-column steps
  const int64_t h = v.m - s;
  const int64_t nI = (h + kTM - 1) / kTM, nJ = (h + kTN - 1) / kTN;
  const int64_t ntiles = 2 * nI * (nI - 1) + nJ;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // tensor-core work issued, and the FP64 update it stands for
    atomicAdd(&flops[KC_FLUSH_TC],
              static_cast<unsigned long long>(2ll * kTM * (kSlices * (kSlices + 1) / 2) * kTN * 16 * KS * ntiles));
    atomicAdd(&flops[KC_COUNT], static_cast<unsigned long long>(2 * static_cast<int64_t>(r) * (h * (h + 1) / 2)));
  }
  if (blockIdx.x >= ntiles) return;
  unsigned char* sbase =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) { tc::mbar_init(&full_bar[i], 1); tc::mbar_init(&empty_bar[i], 1); }
    tc::mbar_init(&tfull_bar, 1);
    tc::mbar_init(&tempty_bar, 4 * 32);
    tc::mbar_init(&drain_bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const int64_t total = my_tiles * KS;

  if (warp == 4) {
    // ---- producer: bulk copies of one 16-column step of all digits of the tile's rows ----
    if (lane == 0) {
      int64_t f = 0;
      bool ok = true;
      for (; f < total; ++f) {
        const int st = static_cast<int>(f % kStages);
        if (f >= kStages && !tc::mbar_wait(&empty_bar[st], static_cast<uint32_t>((f / kStages - 1) & 1), kWaitNs)) {
          ok = false;
          break;
        }
        int64_t I, J;
        tile_ij(blockIdx.x + (f / KS) * gridDim.x, nI, I, J);
        const int kk = static_cast<int>(f % KS);
        unsigned char* sa = sbase + static_cast<size_t>(st) * kStageBytes;
        unsigned char* sb = sa + kStageA;
        tc::mbar_arrive_expect_tx(&full_bar[st], kStageBytes);
#pragma unroll 1
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll 1
          for (int a = 0; a < kSlices; ++a) {
            const int64_t q = static_cast<int64_t>(a) * kKB + 2 * kk + kb;
            tc::bulk_g2s(sa + kb * (kStageA / 2) + a * (kTM * 16), E.Ls + (q * E.R + I * kTM) * 8, kTM * 16,
                         &full_bar[st]);
            tc::bulk_g2s(sb + kb * (kStageB / 2) + a * (kTN * 16), E.Ws + (q * E.R + J * kTN) * 8, kTN * 16,
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
  } else if (warp == 5) {
    // ---- MMA issue: per step, slice a of L against the stacked slices 1 .. 8-a of W ----
    if (lane == 0) {
      const uint32_t s0 = tc::smem_addr(sbase);
      int64_t f = 0;
      bool ok = true;
      for (int64_t n = 0; n < my_tiles && ok; ++n) {
        if (n > 0 && !tc::mbar_wait(&tempty_bar, static_cast<uint32_t>((n - 1) & 1), kWaitNs)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        for (int kk = 0; kk < KS; ++kk, ++f) {
          const int st = static_cast<int>(f % kStages);
          if (!tc::mbar_wait(&full_bar[st], static_cast<uint32_t>((f / kStages) & 1), kWaitNs)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = s0 + st * kStageBytes, sb = sa + kStageA;
          const uint64_t bdesc = tc::smem_desc(sb, kStageB / 2, 128);
#pragma unroll
          for (int a = 0; a < kSlices; ++a) {
            // accumulator of level a+2 (a < 4: first set, columns 32 a; else second set)
            const uint32_t d = tmem + static_cast<uint32_t>(a < 4 ? a * kTN : 8 * kTN + (a - 4) * kTN);
            const uint32_t acc = (kk > 0 || (a != 0 && a != 4)) ? 1u : 0u;
            tc::mma_bf16(d, tc::smem_desc(sa + a * (kTM * 16), kStageA / 2, 128), bdesc,
                         tc::idesc_bf16(kTM, (kSlices - a) * kTN), acc);
          }
          tc::mma_commit(&empty_bar[st]);
        }
        if (!ok) break;
        tc::mma_commit(&tfull_bar);
      }
      if (!ok) abort_flag = 1;
      tc::mma_commit(&drain_bar);               // all MMAs of this CTA done before tensor memory goes
      tc::mbar_wait(&drain_bar, 0, kWaitNs);
    }
  } else {
    // ---- epilogue: warp w reads lanes (rows) 32w .. 32w+31 ----
    const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    for (int64_t n = 0; n < my_tiles; ++n) {
      if (!tc::mbar_wait(&tfull_bar, static_cast<uint32_t>(n & 1), kWaitNs)) {
        abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      int64_t I, J;
      tile_ij(blockIdx.x + n * gridDim.x, nI, I, J);
      long long vh[kTN], vl[kTN];
#pragma unroll
      for (int cg = 0; cg < kTN / 8; ++cg) {
        uint32_t x[8][8], y[4][8];
#pragma unroll
        for (int g = 0; g < 8; ++g) tc::tmem_ld8(trow + g * kTN + cg * 8, x[g]);
#pragma unroll
        for (int g = 0; g < 4; ++g) tc::tmem_ld8(trow + 8 * kTN + g * kTN + cg * 8, y[g]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int g = 0; g < 8; ++g) tc::tmem_keep(x[g]);
#pragma unroll
        for (int g = 0; g < 4; ++g) tc::tmem_keep(y[g]);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          int lv[8];
#pragma unroll
          for (int g = 0; g < 8; ++g) lv[g] = level_int(x[g][e]);
#pragma unroll
          for (int g = 4; g < 8; ++g) lv[g] += level_int(y[g - 4][e]);
          // levels 2..5 and 6..9 in base 256 (each level sum below 2^25 in magnitude)
          vh[cg * 8 + e] = (static_cast<long long>(lv[0]) << 24) + (static_cast<long long>(lv[1]) << 16) +
                           (static_cast<long long>(lv[2]) << 8) + lv[3];
          vl[cg * 8 + e] = (static_cast<long long>(lv[4]) << 24) + (static_cast<long long>(lv[5]) << 16) +
                           (static_cast<long long>(lv[6]) << 8) + lv[7];
        }
      }
      // tensor memory is free for the next tile; the FP64 part overlaps its MMAs
      tc::fence_before_sync();
      tc::mbar_arrive(&tempty_bar);
      const int64_t i = s + I * kTM + warp * 32 + lane;
      if (i < v.m) {
        const int ei = E.eL[i - s];
#pragma unroll
        for (int c = 0; c < kTN; ++c) {
          const int64_t j = s + J * kTN + c;
          if (j <= i) {
            const double upd = combine_to_double(vh[c], vl[c], ei + E.eW[j - s] - 72);
            *v.at(static_cast<int32_t>(i), static_cast<int32_t>(j)) -= upd;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(&S.status[0], ST_TIMEOUT);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

EmulArgs emul_args(void* ws, int64_t cap_rows) {
  EmulArgs E;
  E.cap_rows = cap_rows;
  E.R = digit_pitch(cap_rows);
  const int64_t plane = static_cast<int64_t>(kSlices) * kKB * E.R * 8;
  E.Ls = static_cast<__nv_bfloat16*>(ws);
  E.Ws = E.Ls + plane;
  E.Wv = reinterpret_cast<double*>(E.Ws + plane);
  E.eL = reinterpret_cast<int32_t*>(E.Wv + static_cast<int64_t>(kWindow) * cap_rows);
  E.eW = E.eL + E.R;
  E.cexp = E.eW + E.R;
  return E;
}

}  // namespace

size_t emul_workspace_bytes(int64_t cap_rows) {
  const int64_t R = digit_pitch(cap_rows);
  return 2ull * kSlices * kKB * R * 8 * sizeof(__nv_bfloat16) + kWindow * cap_rows * sizeof(double) +
         2ull * R * sizeof(int32_t) + 2ull * kWindow * sizeof(int32_t) + 512;
}

// Slice and flush for batch entry b (a front factored alone); the kernels return at once unless
// the front's window flush is due this step.
void launch_emul_flush(const FrontTables& T, const FactorSlot& S, double* cbpool, const LargeWork& W,
                       const int32_t* lf, int32_t b, void* ws, int64_t cap_rows, int64_t rows_hint,
                       cudaStream_t st, int num_sms, Timer* timer, unsigned long long* flops) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lf_flush_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kFlushSmem));
    attr_set = true;
  }
  const EmulArgs E = emul_args(ws, cap_rows);
  const int gs = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows_hint + kSRows - 1) / kSRows, num_sms * 4)));
  const int gc = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows_hint + 255) / 256, num_sms * 2)));
  KEP_LAUNCH(timer, KC_SLICE, st, lf_colmax_kernel<<<gc, 256, 0, st>>>(T, S, W, lf, b, E));
  KEP_LAUNCH(timer, KC_SLICE, st, lf_slice_kernel<<<gs, 256, 0, st>>>(T, S, W, lf, b, E));
  KEP_LAUNCH(timer, KC_FLUSH_TC, st,
             lf_flush_tc_kernel<<<num_sms, kFlushThreads, kFlushSmem, st>>>(T, S, cbpool, W, lf, b, E, flops));
}

}  // namespace kep
