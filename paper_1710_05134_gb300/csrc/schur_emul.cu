// FP64-accurate Schur update on the tensor cores (the window flush of the front factorization).
//
// C(i, j) -= sum_c L(i, c) W(j, c), W = L D, for the pivots of one window (rank r <= 256).  GB300
// issues FP64 FMAs at 1/32 of its FP32 rate, so the product is formed from bf16 pieces whose
// products the tensor cores sum exactly (an error-free splitting in the manner of Ozaki et al.):
//
//  * column balancing: column c of L is scaled by 2^{-u_c} and column c of W by 2^{u_c} (u_c from
//    the two columns' largest exponents), which leaves every product unchanged and keeps the
//    spread of D out of the rows;
//  * every row is scaled by a power of two 2^e (|x| < 2^e for all its entries) and written in
//    sign-magnitude base-256 digits, |x| 2^{8-e} = sum_a d_a 256^{1-a}, d_a in [0, 255], a = 1..8,
//    cut from the double's significand with integer shifts (the dropped tail is below 2^-64 of
//    the row's largest entry); each signed digit is exact in bf16;
//  * for each level g = a + b (g <= 9) and each K chunk of 32, the tensor cores sum
//    sum_{a+b=g} sum_c s_a(i, c) t_b(j, c) in FP32; every partial sum is an integer of magnitude
//    at most 8 * 255^2 * 32 < 2^24, so these FP32 sums are exact;
//  * the level sums are combined exactly in two int64 accumulators (levels 2..5 and 6..9) and
//    C(i, j) -= 2^{e_i + f_j} (hi 2^-40 + lo 2^-72) in FP64 once per window.
//
// The only roundings are the one FP64 product L D, the dropped digit tail and the final FP64
// conversion: as accurate as an FP64 rank-r update.
#include <algorithm>

#include <cuda_bf16.h>

#include "kep_device.cuh"

namespace kep {

namespace {

constexpr int kSlices = 8;
constexpr int kETile = 64;                    // CTA tile (rows x columns)
constexpr int kEK = 32;                       // K chunk per shared-memory stage
constexpr int kEPitch = kEK + 8;              // bf16 per shared row (conflict-free fragment loads)
constexpr int kEThreads = 128;                // 4 warps, 32 x 32 each
constexpr size_t kEmulSmem = 2ull * kSlices * kETile * kEPitch * sizeof(__nv_bfloat16);

struct EmulArgs {
  __nv_bfloat16* Ls;   // [kSlices][rows][kWindow] signed digits of the balanced, scaled L rows
  __nv_bfloat16* Ws;   // same for W
  double* Wv;          // [kWindow][rows] W = L D (column-major, like L)
  int32_t* eL;         // [rows] row scale exponents
  int32_t* eW;
  int32_t* cexp;       // [2][kWindow] largest biased exponent of |L(., c)| and |W(., c)|
  int64_t cap_rows;
};

KEP_D double pow2(int e) {
  return __longlong_as_double(static_cast<long long>(e + 1023) << 52);
}

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

// 64-bit fixed point floor(|x| 2^{-u} 2^{8-e} 2^56) of a normal double x (0 for zero/subnormal)
KEP_D unsigned long long fixed56(double x, int u, int e) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bits >> 52) & 0x7ff);
  if (E == 0) return 0ull;
  const unsigned long long M = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = E - 1011 - u - e;             // value M 2^{E-1075} scaled by 2^{-u+8-e+56}
  if (sh >= 0) return M << sh;                 // sh <= 11 because the scaled value is below 256
  if (sh <= -64) return 0ull;
  return M >> (-sh);
}

KEP_D __nv_bfloat16 digit_bf16(unsigned d, bool neg) {
  const float f = __uint2float_rn(d);          // d <= 255: exact, low 16 bits of f are zero
  const unsigned short h = static_cast<unsigned short>(__float_as_uint(f) >> 16) | (neg && d ? 0x8000 : 0);
  return __ushort_as_bfloat16(h);
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

// Pass 2: per row, the scale exponent of the balanced row, then the eight signed digits of every
// entry, staged through shared memory so each (digit, row) segment is stored contiguously.
constexpr int kSRows = 32;                     // rows per CTA
__global__ void __launch_bounds__(256) lf_slice_kernel(FrontTables T, FactorSlot S, LargeWork W, const int32_t* lf,
                                                       int32_t b, EmulArgs E) {
  __shared__ __nv_bfloat16 sd[2][kSlices][kSRows][kEK + 2];
  __shared__ int se[2][kSRows];
  if (W.done[b] || !W.flush[b]) return;
  const int32_t t = lf[b];
  const int32_t d_in = S.d_in[t];
  const int32_t m = T.m_sym[t] + d_in;
  const int32_t c0 = W.ws[b], c1 = W.kend[b], s = W.we[b];
  const int32_t r = c1 - c0;
  if (r <= 0 || s >= m) return;
  const int32_t rc = (r + kEK - 1) / kEK * kEK;
  const double* L = S.F + T.front_off[t];
  const int64_t ld = T.m_alloc[t];
  const int64_t rows = m - s;
  const int64_t stride = E.cap_rows * kWindow;   // between digits
  const int lr = threadIdx.x % kSRows;           // row within the CTA's block (loads: coalesced)
  const int lc = threadIdx.x / kSRows;           // 8 column lanes
  for (int64_t rb = static_cast<int64_t>(blockIdx.x) * kSRows; rb < rows; rb += static_cast<int64_t>(gridDim.x) * kSRows) {
    const int64_t row = rb + lr;
    const bool ok = row < rows;
    // row exponents of the balanced entries
    int ex = 0, ey = 0;
    if (ok)
      for (int32_t c = lc; c < r; c += 256 / kSRows) {
        const int u = balance_shift(E, c);
        const int bx = bexp(L[static_cast<int64_t>(c0 + c) * ld + s + row]);
        const int by = bexp(E.Wv[static_cast<int64_t>(c) * E.cap_rows + row]);
        if (bx) ex = max(ex, bx - u);
        if (by) ey = max(ey, by + u);
      }
    __syncthreads();
    if (lc == 0) { se[0][lr] = 0; se[1][lr] = 0; }
    __syncthreads();
    atomicMax(&se[0][lr], ex);
    atomicMax(&se[1][lr], ey);
    __syncthreads();
    const int el = se[0][lr] ? se[0][lr] - 1022 : 0;      // |x 2^-u| < 2^el for the whole row
    const int ew = se[1][lr] ? se[1][lr] - 1022 : 0;
    if (ok && lc == 0) { E.eL[row] = el; E.eW[row] = ew; }
    for (int32_t kc = 0; kc < rc; kc += kEK) {
      for (int32_t cc = lc; cc < kEK; cc += 256 / kSRows) {
        const int32_t c = kc + cc;
        double x = 0.0, y = 0.0;
        int u = 0;
        if (ok && c < r) {
          u = balance_shift(E, c);
          x = L[static_cast<int64_t>(c0 + c) * ld + s + row];
          y = E.Wv[static_cast<int64_t>(c) * E.cap_rows + row];
        }
        const unsigned long long X = fixed56(x, u, el), Y = fixed56(y, -u, ew);
        const bool nx = x < 0.0, ny = y < 0.0;
#pragma unroll
        for (int a = 0; a < kSlices; ++a) {
          sd[0][a][lr][cc] = digit_bf16(static_cast<unsigned>((X >> (56 - 8 * a)) & 0xff), nx);
          sd[1][a][lr][cc] = digit_bf16(static_cast<unsigned>((Y >> (56 - 8 * a)) & 0xff), ny);
        }
      }
      __syncthreads();
      // store: 2 operands x 8 digits x 32 rows x 32 columns, 4 bytes per thread-store
      for (int32_t e = threadIdx.x; e < 2 * kSlices * kSRows * (kEK / 2); e += blockDim.x) {
        const int32_t pair = e % (kEK / 2);
        const int32_t rr = (e / (kEK / 2)) % kSRows;
        const int32_t a = (e / (kEK / 2 * kSRows)) % kSlices;
        const int32_t which = e / (kEK / 2 * kSRows * kSlices);
        const int64_t grow = rb + rr;
        if (grow >= rows) continue;
        const __nv_bfloat162 v2 = __halves2bfloat162(sd[which][a][rr][2 * pair], sd[which][a][rr][2 * pair + 1]);
        __nv_bfloat16* dst = (which == 0 ? E.Ls : E.Ws) + a * stride + grow * kWindow + kc + 2 * pair;
        *reinterpret_cast<__nv_bfloat162*>(dst) = v2;
      }
      __syncthreads();
    }
  }
}

KEP_D uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__global__ void __launch_bounds__(kEThreads, 2) lf_flush_emul_kernel(FrontTables T, FactorSlot S, double* cbpool,
                                                                     LargeWork W, const int32_t* lf, int32_t b,
                                                                     EmulArgs E, unsigned long long* flops) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* Bs = As + kSlices * kETile * kEPitch;
  if (W.done[b] || !W.flush[b]) return;
  if (blockIdx.x == 0)                        // column exponents are used up: clear for the next window
    for (int32_t c = threadIdx.x; c < 2 * kWindow; c += blockDim.x) E.cexp[c] = 0;
  const int32_t t = lf[b];
  const int32_t d_in = S.d_in[t];
  const FrontView v = front_view(T, S, cbpool, t, d_in);
  const int32_t c0 = W.ws[b], c1 = W.kend[b], s = W.we[b];
  const int32_t r = c1 - c0;
  if (r <= 0 || s >= v.m) return;
  const int32_t rc = (r + kEK - 1) / kEK * kEK;
  const int64_t stride = E.cap_rows * kWindow;
  // lower-triangle tiles of [s, m) with blocks split at p (L storage / contribution block)
  const int32_t nL = s < v.p ? (v.p - s + kETile - 1) / kETile : 0;
  const int32_t base2 = s > v.p ? s : v.p;
  const int32_t nR = nL + (v.m > base2 ? (v.m - base2 + kETile - 1) / kETile : 0);
  auto blo = [&](int32_t q) { return q < nL ? s + q * kETile : base2 + (q - nL) * kETile; };
  auto bhi = [&](int32_t q) { return q < nL ? min(s + (q + 1) * kETile, v.p) : min(base2 + (q - nL + 1) * kETile, v.m); };
  const int64_t ntiles = static_cast<int64_t>(nR) * (nR + 1) / 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // tensor-core work issued: every tile, every K chunk, every (level, pair) product
    constexpr int64_t kPairs = kSlices * (kSlices + 1) / 2;
    atomicAdd(&flops[KC_FLUSH_TC], static_cast<unsigned long long>(2 * kPairs * rc * ntiles * kETile * kETile));
    // the FP64 update it stands for
    const int64_t h = v.m - s;
    atomicAdd(&flops[KC_COUNT], static_cast<unsigned long long>(2 * static_cast<int64_t>(r) * (h * (h + 1) / 2)));
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int wr = warp >> 1, wc = warp & 1;
  const int gq = lane >> 2, tq = lane & 3;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int32_t bi = static_cast<int32_t>((sqrt(8.0 * static_cast<double>(tile) + 1.0) - 1.0) * 0.5);
    while (static_cast<int64_t>(bi) * (bi + 1) / 2 > tile) --bi;
    while (static_cast<int64_t>(bi + 1) * (bi + 2) / 2 <= tile) ++bi;
    const int32_t bj = static_cast<int32_t>(tile - static_cast<int64_t>(bi) * (bi + 1) / 2);
    const int32_t I0 = blo(bi), I1 = bhi(bi), J0 = blo(bj), J1 = bhi(bj);
    long long Vh[2][4][4], Vl[2][4][4];       // levels 2..5 and 6..kSlices+1, exact
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) { Vh[mi][ni][e] = 0; Vl[mi][ni][e] = 0; }
    for (int32_t kc = 0; kc < rc; kc += kEK) {
      __syncthreads();
      // stage the kSlices pieces of rows I0.. and J0.. for columns kc .. kc+32 (16-byte loads)
      for (int32_t e = threadIdx.x; e < 2 * kSlices * kETile * (kEK / 8); e += blockDim.x) {
        const int32_t part = e % (kEK / 8);
        const int32_t rowi = (e / (kEK / 8)) % kETile;
        const int32_t sl = (e / (kEK / 8 * kETile)) % kSlices;
        const int32_t which = e / (kEK / 8 * kETile * kSlices);
        const int32_t g0 = which == 0 ? I0 : J0, g1 = which == 0 ? I1 : J1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (g0 + rowi < g1) {
          const __nv_bfloat16* src = (which == 0 ? E.Ls : E.Ws) + sl * stride +
                                     static_cast<int64_t>(g0 + rowi - s) * kWindow + kc + part * 8;
          val = *reinterpret_cast<const uint4*>(src);
        }
        __nv_bfloat16* dst = (which == 0 ? As : Bs) + (sl * kETile + rowi) * kEPitch + part * 8;
        *reinterpret_cast<uint4*>(dst) = val;
      }
      __syncthreads();
#pragma unroll 1
      for (int g = 2; g <= kSlices + 1; ++g) {
        float acc[2][4][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
          for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
        const int alo = g - kSlices > 1 ? g - kSlices : 1, ahi = g - 1 < kSlices ? g - 1 : kSlices;
#pragma unroll 1
        for (int a = alo; a <= ahi; ++a) {
          const __nv_bfloat16* Aa = As + (a - 1) * kETile * kEPitch;
          const __nv_bfloat16* Bb = Bs + (g - a - 1) * kETile * kEPitch;
#pragma unroll
          for (int ks = 0; ks < kEK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
              const __nv_bfloat16* p0 = Aa + (wr * 32 + mi * 16 + gq) * kEPitch + ks + tq * 2;
              af[mi][0] = lds32(p0);
              af[mi][1] = lds32(p0 + 8 * kEPitch);
              af[mi][2] = lds32(p0 + 8);
              af[mi][3] = lds32(p0 + 8 * kEPitch + 8);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
              const __nv_bfloat16* q0 = Bb + (wc * 32 + ni * 8 + gq) * kEPitch + ks + tq * 2;
              bf[ni][0] = lds32(q0);
              bf[ni][1] = lds32(q0 + 8);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
              for (int ni = 0; ni < 4; ++ni)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                    "{%8,%9}, {%0,%1,%2,%3};"
                    : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
                    : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bf[ni][0]),
                      "r"(bf[ni][1]));
          }
        }
        // exact integer level sums into the two accumulators
        if (g <= 5) {
          const long long mul = 1ll << (8 * (5 - g));
#pragma unroll
          for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
              for (int e = 0; e < 4; ++e) Vh[mi][ni][e] += static_cast<long long>(__float2int_rz(acc[mi][ni][e])) * mul;
        } else {
          const long long mul = 1ll << (8 * (kSlices + 1 - g));
#pragma unroll
          for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
              for (int e = 0; e < 4; ++e) Vl[mi][ni][e] += static_cast<long long>(__float2int_rz(acc[mi][ni][e])) * mul;
        }
      }
    }
    // C(i, j) -= 2^{e_i + f_j} (Vh 2^-40 + Vl 2^-8(kSlices+1))
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int32_t i = I0 + wr * 32 + mi * 16 + gq + (e >= 2 ? 8 : 0);
          const int32_t j = J0 + wc * 32 + ni * 8 + tq * 2 + (e & 1);
          if (i < I1 && j < J1 && i >= j) {
            const int ex = E.eL[i - s] + E.eW[j - s];
            *v.at(i, j) -= __ll2double_rn(Vh[mi][ni][e]) * pow2(ex - 40) +
                           __ll2double_rn(Vl[mi][ni][e]) * pow2(ex - 8 * (kSlices + 1));
          }
        }
  }
}

}  // namespace

size_t emul_workspace_bytes(int64_t cap_rows) {
  return 2ull * kSlices * cap_rows * kWindow * sizeof(__nv_bfloat16) + kWindow * cap_rows * sizeof(double) +
         2ull * cap_rows * sizeof(int32_t) + 2ull * kWindow * sizeof(int32_t) + 512;
}

// Slice and flush for batch entry b (a front factored alone); both kernels return at once unless
// the front's window flush is due this step.
void launch_emul_flush(const FrontTables& T, const FactorSlot& S, double* cbpool, const LargeWork& W,
                       const int32_t* lf, int32_t b, void* ws, int64_t cap_rows, int64_t rows_hint,
                       cudaStream_t st, int num_sms, Timer* timer, unsigned long long* flops) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lf_flush_emul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kEmulSmem));
    attr_set = true;
  }
  EmulArgs E;
  E.cap_rows = cap_rows;
  E.Ls = static_cast<__nv_bfloat16*>(ws);
  E.Ws = E.Ls + static_cast<int64_t>(kSlices) * cap_rows * kWindow;
  E.Wv = reinterpret_cast<double*>(E.Ws + static_cast<int64_t>(kSlices) * cap_rows * kWindow);
  E.eL = reinterpret_cast<int32_t*>(E.Wv + static_cast<int64_t>(kWindow) * cap_rows);
  E.eW = E.eL + cap_rows;
  E.cexp = E.eW + cap_rows;
  const int gs = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows_hint + kSRows - 1) / kSRows, num_sms * 8)));
  const int gc = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows_hint + 255) / 256, num_sms * 2)));
  KEP_LAUNCH(timer, KC_SLICE, st, lf_colmax_kernel<<<gc, 256, 0, st>>>(T, S, W, lf, b, E));
  KEP_LAUNCH(timer, KC_SLICE, st, lf_slice_kernel<<<gs, 256, 0, st>>>(T, S, W, lf, b, E));
  KEP_LAUNCH(timer, KC_FLUSH_TC, st,
             lf_flush_emul_kernel<<<num_sms * 2, kEThreads, kEmulSmem, st>>>(T, S, cbpool, W, lf, b, E, flops));
}

}  // namespace kep
