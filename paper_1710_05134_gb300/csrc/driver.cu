// Three-stage k-th eigenpair driver (Algorithm 4, Section 3.4) on the GPU path.
//
//  Stage 1 (Algorithm 2): factor B (task (ii) of Section 4.3), run the generalized Lanczos process
//    A V_j = B V_j T_j + B v_{j+1} beta_j e_j^T (Eq. 2.2, V_j B-orthonormal, w = B^{-1} A v_j), take
//    sigma^(j) = theta_1^(j) if k <= nu^(j-1) else theta_j^(j) and factor A - sigma^(j) B, until nu
//    brackets k at j != 1.
//  Stage 2 (Algorithm 1'): bisect [sigma_l, sigma_u) until nu_u - nu_l <= m_max.
//  Stage 3 (Algorithm 3): factor A - sigma B at the midpoint and run the shift-and-invert Lanczos
//    process of Eq. 2.5.  It is carried out for V = B^{-1} V~ (so V is B-orthonormal and only
//    (A - sigma B)^{-1} and products with B are needed): (A - sigma B)^{-1} B V_j = V_j T~_j +
//    v_{j+1} beta~_j e_j^T, the same T~_j.  Ritz values lambda_i = sigma + 1/theta~_i (Eq. 2.7); the
//    modified Ritz vectors x_{i,2} = (A - sigma B)^{-1} V~_j y~_i (Eq. 2.9) follow without a solve from
//    the decomposition: x_{i,2} = theta~_i V_j y~_i + v_{j+1} beta~_j (e_j^T y~_i) (proof of
//    Proposition 1).  Bounds eta_i (Proposition 3, Eq. 3.1), inclusion (3.3), disjointness (3.4),
//    residual and relative difference (3.5) decide convergence; the residual uses the identity
//    r_{i,2} = -B v_{j+1} (beta~_j e_j^T y~_i / theta~_i) (Eq. 2.12) while iterating and is recomputed
//    explicitly with the sparse products before the result is accepted.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "kep_ctx.h"
#include "kep_vec.h"

namespace kep {

// ----------------------------------------------------------------------------------------------
// Gershgorin bounds of A and B (full symmetric CSR): per block the extremes of a_ii -+ r_i and
// b_ii -+ s_i (r_i, s_i the off-diagonal absolute row sums) as [4][nblocks] = min lo_A, max hi_A,
// min lo_B, max hi_B
// ----------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gershgorin_kernel(int64_t n, const int64_t* rp, const int32_t* ci,
                                                         const double* a, const double* b, double* out) {
  __shared__ double red[4][8];
  double loA = INFINITY, hiA = -INFINITY, loB = INFINITY, hiB = -INFINITY;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double da = 0.0, db = 0.0, ra = 0.0, rb = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] == i) { da = a[p]; db = b[p]; }
      else { ra += fabs(a[p]); rb += fabs(b[p]); }
    }
    loA = fmin(loA, da - ra); hiA = fmax(hiA, da + ra);
    loB = fmin(loB, db - rb); hiB = fmax(hiB, db + rb);
  }
  for (int o = 16; o > 0; o >>= 1) {
    loA = fmin(loA, __shfl_xor_sync(0xffffffffu, loA, o));
    hiA = fmax(hiA, __shfl_xor_sync(0xffffffffu, hiA, o));
    loB = fmin(loB, __shfl_xor_sync(0xffffffffu, loB, o));
    hiB = fmax(hiB, __shfl_xor_sync(0xffffffffu, hiB, o));
  }
  const int w = threadIdx.x / 32;
  if (threadIdx.x % 32 == 0) { red[0][w] = loA; red[1][w] = hiA; red[2][w] = loB; red[3][w] = hiB; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < 8; ++q) {
      red[0][0] = fmin(red[0][0], red[0][q]); red[1][0] = fmax(red[1][0], red[1][q]);
      red[2][0] = fmin(red[2][0], red[2][q]); red[3][0] = fmax(red[3][0], red[3][q]);
    }
    for (int k = 0; k < 4; ++k) out[k * gridDim.x + blockIdx.x] = red[k][0];
  }
}

// ----------------------------------------------------------------------------------------------
// symmetric tridiagonal eigenproblem: implicit QR steps with Wilkinson shifts, applied as Givens
// rotations to a dense copy (m is at most a few hundred here), rotations accumulated into z
// ----------------------------------------------------------------------------------------------
bool tridiag_eigen(int m, const double* d, const double* e, double* w, double* z) {
  std::vector<double> T(static_cast<size_t>(m) * m, 0.0);
  auto t = [&](int i, int j) -> double& { return T[static_cast<size_t>(j) * m + i]; };
  for (int i = 0; i < m; ++i) {
    t(i, i) = d[i];
    if (i + 1 < m) { t(i + 1, i) = e[i]; t(i, i + 1) = e[i]; }
  }
  for (int i = 0; i < m * m; ++i) z[i] = 0.0;
  for (int i = 0; i < m; ++i) z[static_cast<size_t>(i) * m + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  auto small = [&](int q) {   // is the sub-diagonal entry (q, q-1) negligible?
    double s = std::fabs(t(q, q)) + std::fabs(t(q - 1, q - 1));
    return std::fabs(t(q, q - 1)) <= eps * s || std::fabs(t(q, q - 1)) < 1e-300;
  };
  int q = m - 1;
  int iter = 0;
  const int max_iter = 60 * std::max(m, 1);
  while (q > 0) {
    if (small(q)) { t(q, q - 1) = t(q - 1, q) = 0.0; --q; continue; }
    if (++iter > max_iter) return false;
    int p = q - 1;
    while (p > 0 && !small(p)) --p;
    if (p > 0) { t(p, p - 1) = t(p - 1, p) = 0.0; }
    // Wilkinson shift: eigenvalue of the trailing 2x2 block closer to t(q, q)
    const double a = t(q - 1, q - 1), b = t(q, q - 1), c = t(q, q);
    const double delta = 0.5 * (a - c);
    const double sg = delta >= 0 ? 1.0 : -1.0;
    const double mu = c - b * b / (delta + sg * std::sqrt(delta * delta + b * b));
    double x = t(p, p) - mu, y = t(p + 1, p);
    for (int k = p; k < q; ++k) {
      const double r = std::hypot(x, y);
      const double cs = r == 0.0 ? 1.0 : x / r, sn = r == 0.0 ? 0.0 : y / r;
      const int lo = std::max(p, k - 1), hi = std::min(q, k + 2);
      for (int col = lo; col <= hi; ++col) {      // rows k, k+1
        const double u = t(k, col), v = t(k + 1, col);
        t(k, col) = cs * u + sn * v;
        t(k + 1, col) = -sn * u + cs * v;
      }
      for (int row = lo; row <= hi; ++row) {      // columns k, k+1
        const double u = t(row, k), v = t(row, k + 1);
        t(row, k) = cs * u + sn * v;
        t(row, k + 1) = -sn * u + cs * v;
      }
      for (int row = 0; row < m; ++row) {         // accumulate Z <- Z G^T
        double* zk = z + static_cast<size_t>(k) * m;
        double* zk1 = z + static_cast<size_t>(k + 1) * m;
        const double u = zk[row], v = zk1[row];
        zk[row] = cs * u + sn * v;
        zk1[row] = -sn * u + cs * v;
      }
      if (k + 1 < q) { x = t(k + 1, k); y = t(k + 2, k); }
    }
  }
  // sort ascending
  std::vector<int> idx(m);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return t(i, i) < t(j, j); });
  std::vector<double> zc(z, z + static_cast<size_t>(m) * m);
  for (int i = 0; i < m; ++i) {
    w[i] = t(idx[i], idx[i]);
    std::memcpy(z + static_cast<size_t>(i) * m, zc.data() + static_cast<size_t>(idx[i]) * m, sizeof(double) * m);
  }
  return true;
}

namespace {

struct Driver {
  int64_t cap_cols = 0;
  double* V = nullptr;      // n x cap_cols, B-orthonormal basis
  double* BV = nullptr;     // B * V
  double* w = nullptr;      // work vectors
  double* u = nullptr;
  double* u2 = nullptr;
  double* coef = nullptr;   // device coefficients (cap_cols)
  double* partial = nullptr;
  int nblocks = 0;
  double* cg = nullptr;     // 3 n: residual, direction, B times direction (B-solves by CG)
};

// splitmix64 (Steele, Lea, Flood 2014) as a counter-based generator; Box-Muller for N(0, 1).
uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

void gaussian_vector(uint64_t seed, int64_t n, double* out) {
  const double two_pi = 6.283185307179586;
  for (int64_t i = 0; i < n; i += 2) {
    const uint64_t r1 = splitmix64(seed * 0x100000001b3ull + 2 * static_cast<uint64_t>(i));
    const uint64_t r2 = splitmix64(seed * 0x100000001b3ull + 2 * static_cast<uint64_t>(i) + 1);
    const double u1 = (static_cast<double>(r1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = static_cast<double>(r2 >> 11) * (1.0 / 9007199254740992.0);
    const double rad = std::sqrt(-2.0 * std::log(u1));
    out[i] = rad * std::cos(two_pi * u2);
    if (i + 1 < n) out[i + 1] = rad * std::sin(two_pi * u2);
  }
}

using clock_ = std::chrono::steady_clock;
double seconds_since(clock_::time_point t0) {
  return std::chrono::duration<double>(clock_::now() - t0).count();
}

}  // namespace
}  // namespace kep

using namespace kep;

void kep_ctx::driver_release() {
  Driver* d = static_cast<Driver*>(driver);
  if (!d) return;
  cudaFree(d->V); cudaFree(d->BV); cudaFree(d->w); cudaFree(d->u); cudaFree(d->u2);
  cudaFree(d->coef); cudaFree(d->partial); cudaFree(d->cg);
  delete d;
  driver = nullptr;
}

namespace {

#define DTRY(x) do { kep_status _s = (x); if (_s != KEP_OK) return _s; } while (0)
#define CTRY(x) do { if ((x) != cudaSuccess) return KEP_ERR_CUDA; } while (0)

struct Run {
  kep_ctx* c;
  Driver* d;
  VecOps ops;
  VecOps opsh;          // over the first herm_n rows (halves of an embedded Hermitian vector)
  int64_t n;
  double norm_a;
  kep_report rep{};

  double* col(double* base, int64_t j) { return base + j * n; }

  kep_status sync() { return cudaStreamSynchronize(c->stream) == cudaSuccess ? KEP_OK : KEP_ERR_CUDA; }

  kep_status to_host(double* h, const double* dptr, int64_t cnt) {
    CTRY(cudaMemcpyAsync(h, dptr, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
    return sync();
  }

  // out = V(:, 0:ncol)^T w on the host
  kep_status dots(const double* Vb, int32_t ncol, const double* wv, double* out) {
    ops.dots(Vb, n, ncol, wv, d->coef);
    return to_host(out, d->coef, ncol);
  }

  // w -= Vb(:, 0:ncol) coef (coef from the host)
  kep_status sub_combine(const double* Vb, int32_t ncol, const double* coef_h, double* wv) {
    CTRY(cudaMemcpyAsync(d->coef, coef_h, sizeof(double) * ncol, cudaMemcpyHostToDevice, c->stream));
    ops.combine(Vb, n, ncol, d->coef, -1.0, 1.0, wv);
    return KEP_OK;
  }

  // nu(sigma) with slot 0 (a shift exactly at an eigenvalue is nudged upward)
  kep_status nu_at(double& sigma, int64_t& nu) {
    for (int attempt = 0; attempt < 8; ++attempt) {
      kep_inertia in{};
      kep_status st = ctx_factor(c, 0, 1.0, -sigma, &in);
      rep.n_factor++;
      if (st == KEP_OK) { nu = in.neg; return KEP_OK; }
      if (st != KEP_ERR_SINGULAR) return st;
      sigma += 8.0 * 2.220446049250313e-16 * std::max(1.0, norm_a) * std::max(1.0, std::fabs(sigma)) * (attempt + 1);
    }
    return KEP_ERR_SINGULAR;
  }

  // Slot of B's factor: slot 1 while a second factor fits on the device next to slot 0;
  // otherwise B shares slot 0 with the factorizations of A - sigma B and is factored again
  // whenever a B-solve finds slot 0 holding another matrix (at most once per Algorithm 2 step).
  int bslot = 1;

  kep_status choose_bslot(int32_t policy) {
    if (policy == KEP_BFACTOR_SHARED) { bslot = 0; return KEP_OK; }
    if (policy == KEP_BFACTOR_OWN || c->slot_ready[1]) { bslot = 1; return KEP_OK; }
    size_t free_b = 0, total_b = 0;
    CTRY(cudaMemGetInfo(&free_b, &total_b));
    // a second slot must fit beside what the shifted factorizations still allocate: their own slot
    // (allocated at the first factorization) and the tensor-core workspace (at most 24 GB)
    const Plan& P = c->plan;
    const double slot = 8.0 * static_cast<double>(P.front_total) + 8.0 * static_cast<double>(P.vec_total) +
                        17.0 * static_cast<double>(P.piv_total);
    double need = slot + (2ll << 30);
    if (!c->slot_ready[0]) need += slot;
    if (c->emul_bytes == 0) need += static_cast<double>(24ll << 30);
    bslot = static_cast<double>(free_b) > need ? 1 : 0;
    return KEP_OK;
  }

  bool b_factored() const {
    const FactorSlot& S = c->slot[bslot];
    return c->slot_ready[bslot] && S.valid && S.ca == 0.0 && S.cb == 1.0;
  }

  kep_status factor_B() {
    kep_inertia in{};
    kep_status st = ctx_factor(c, bslot, 0.0, 1.0, &in);
    rep.n_factor++;
    if (st == KEP_ERR_SINGULAR) return KEP_ERR_NOT_SPD;
    if (st != KEP_OK) return st;
    if (in.neg != 0 || in.zero != 0) return KEP_ERR_NOT_SPD;
    b_spd = true;
    return KEP_OK;
  }

  bool b_spd = false;       // B's factorization showed it positive definite

  // x = B^{-1} b by conjugate gradients (B is positive definite): the B-solves of a shared slot
  // once the slot holds another matrix.  Stops at ||b - B x||_2 <= 1e-14 ||b||_2; false (x not
  // usable) when that takes more than 500 iterations.
  kep_status cg_B(const double* b, double* x, bool& converged) {
    converged = false;
    if (!d->cg) {
      if (cudaMalloc(&d->cg, sizeof(double) * 3 * n) != cudaSuccess) { cudaGetLastError(); return KEP_OK; }
    }
    double* r = d->cg;
    double* pdir = d->cg + n;
    double* q = d->cg + 2 * n;
    CTRY(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    CTRY(cudaMemcpyAsync(pdir, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    CTRY(cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
    double rr = 0;
    DTRY(dots(r, 1, r, &rr));
    const double stop = 1e-28 * rr;
    for (int it = 0; it < 500; ++it) {
      if (rr <= stop) { converged = true; return KEP_OK; }
      DTRY(ctx_spmv_dev(c, pdir, nullptr, q));
      double pq = 0;
      DTRY(dots(pdir, 1, q, &pq));
      if (!(pq > 0)) return KEP_OK;
      const double alpha = rr / pq;
      ops.axpby(alpha, pdir, 1.0, x);
      ops.axpby(-alpha, q, 1.0, r);
      double rr1 = 0;
      DTRY(dots(r, 1, r, &rr1));
      ops.axpby(1.0, r, rr1 / rr, pdir);
      rr = rr1;
    }
    converged = rr <= stop;
    return KEP_OK;
  }

  kep_status solve_B(const double* b, double* x) {
    if (!b_factored() && bslot == 0 && b_spd) {
      // the shared slot holds A - sigma B: conjugate gradients instead of factoring B again
      bool ok = false;
      DTRY(cg_B(b, x, ok));
      if (ok) return KEP_OK;
    }
    if (!b_factored()) DTRY(factor_B());   // shared slot, or a re-plan of the storage dropped it
    return ctx_solve_dev(c, bslot, b, x);
  }

  // B-normalize column j of V (given in V(:, j)), fill BV(:, j); returns the B-norm
  kep_status b_normalize(int64_t j, double& nrm) {
    DTRY(ctx_spmv_dev(c, col(d->V, j), nullptr, col(d->BV, j)));
    double s = 0;
    DTRY(dots(col(d->V, j), 1, col(d->BV, j), &s));
    if (!(s > 0)) return KEP_ERR_NOT_SPD;
    nrm = std::sqrt(s);
    ops.axpby(0.0, col(d->V, j), 1.0 / nrm, col(d->V, j));
    ops.axpby(0.0, col(d->BV, j), 1.0 / nrm, col(d->BV, j));
    return KEP_OK;
  }

  // full reorthogonalization of w against V(:, 0:ncol) in the B inner product, twice.  For a
  // Hermitian pencil (vectors [re; im] of its real embedding) also against J V, J [u; v] = [-v; u]
  // (multiplication by i): the complex Gram-Schmidt of the complex Lanczos process written in
  // real arithmetic.  Without it rounding lets the second copy of each (doubled) eigenvalue of the
  // embedding into the basis.
  kep_status reorth(int32_t ncol, double* wv, std::vector<double>& tmp) {
    tmp.resize(ncol);
    std::vector<double> t2;
    for (int pass = 0; pass < 2; ++pass) {
      DTRY(dots(d->BV, ncol, wv, tmp.data()));
      DTRY(sub_combine(d->V, ncol, tmp.data(), wv));
      if (c->herm_n) {
        const int64_t h = c->herm_n;
        t2.resize(ncol);
        // (J BV_j) . w = BV_j(top) . w(bottom) - BV_j(bottom) . w(top)
        opsh.dots(d->BV, n, ncol, wv + h, d->coef);
        DTRY(to_host(tmp.data(), d->coef, ncol));
        opsh.dots(d->BV + h, n, ncol, wv, d->coef);
        DTRY(to_host(t2.data(), d->coef, ncol));
        for (int32_t q = 0; q < ncol; ++q) tmp[q] -= t2[q];
        // w -= (J V) h: w(top) += V(bottom) h, w(bottom) -= V(top) h
        CTRY(cudaMemcpyAsync(d->coef, tmp.data(), sizeof(double) * ncol, cudaMemcpyHostToDevice, c->stream));
        opsh.combine(d->V + h, n, ncol, d->coef, 1.0, 1.0, wv);
        opsh.combine(d->V, n, ncol, d->coef, -1.0, 1.0, wv + h);
        DTRY(sync());                                  // tmp (host) is reused by the next pass
      }
    }
    return KEP_OK;
  }
};

}  // namespace

extern "C" kep_status kep_multisection_points(double lo, double hi, int32_t nshift, double* sigmas) {
  if (!sigmas || nshift < 1 || !(lo < hi)) return KEP_ERR_INVALID;
  if (nshift == 1) { sigmas[0] = 0.5 * (lo + hi); return KEP_OK; }
  for (int32_t q = 1; q <= nshift; ++q) sigmas[q - 1] = lo + (hi - lo) * static_cast<double>(q) / (nshift + 1);
  return KEP_OK;
}

extern "C" kep_status kep_multisection_update(int64_t k, int32_t count, const double* sigmas, const int64_t* nus,
                                              double* lo, double* hi, int64_t* nu_lo, int64_t* nu_hi) {
  if (!sigmas || !nus || !lo || !hi || !nu_lo || !nu_hi || count < 1) return KEP_ERR_INVALID;
  if (!(*nu_lo < k && k <= *nu_hi)) return KEP_ERR_INVALID;
  double plo = *lo, phi = *hi;
  int64_t pnl = *nu_lo, pnh = *nu_hi;
  for (int32_t q = 0; q < count; ++q) {
    // counts must not decrease with sigma, and the shifts must lie inside the bracket, in order
    const double s = sigmas[q];
    if (!(s >= plo && s <= phi) || nus[q] < pnl || nus[q] > pnh) return KEP_ERR_INVALID;
    if (k <= nus[q]) { phi = s; pnh = nus[q]; break; }
    plo = s; pnl = nus[q];
  }
  *lo = plo; *hi = phi; *nu_lo = pnl; *nu_hi = pnh;
  return KEP_OK;
}

// Interpolating shift rule (the root-finder variant of Algorithm 1', Sections 2.1 and 5).
static bool interp_bracket_ok(const kep_interp_state* st, int64_t k) {
  return st->lo < st->hi && st->nu_lo < k && k <= st->nu_hi && st->w_lo < st->w_hi;
}

extern "C" kep_status kep_interp_init(int64_t k, double lo, double hi, int64_t nu_lo, int64_t nu_hi,
                                      kep_interp_state* st) {
  if (!st || !(lo < hi) || !(nu_lo < k && k <= nu_hi)) return KEP_ERR_INVALID;
  *st = kep_interp_state{};
  st->lo = lo; st->hi = hi; st->nu_lo = nu_lo; st->nu_hi = nu_hi;
  st->w_lo = static_cast<double>(nu_lo); st->w_hi = static_cast<double>(nu_hi);
  st->width[0] = nu_hi - nu_lo;
  st->nwidth = 1;
  return KEP_OK;
}

extern "C" kep_status kep_interp_point(const kep_interp_state* st, int64_t k, int64_t m_max, double* sigma) {
  if (!st || !sigma || m_max < 1 || !interp_bracket_ok(st, k)) return KEP_ERR_INVALID;
  const double lo = st->lo, hi = st->hi;
  if (st->bisect_next) {
    *sigma = 0.5 * (lo + hi);
    return (*sigma > lo && *sigma < hi) ? KEP_OK : KEP_ERR_CLUSTER;
  }
  const int64_t h = std::max<int64_t>(1, m_max / 4);
  // move the end that is farther from k in count, to inside the final window
  const bool lower_end = (k - st->nu_lo) > (st->nu_hi - k);
  double target = static_cast<double>(lower_end ? k - h : k - 1 + h);
  target = std::min(std::max(target, st->w_lo + 0.5), st->w_hi - 0.5);
  const double f = (target - st->w_lo) / (st->w_hi - st->w_lo);
  const double span = hi - lo;
  const double margin = span / 1048576.0;
  double s = lo + f * span;
  s = std::max(s, lo + margin);
  s = std::min(s, hi - margin);
  if (!(s > lo && s < hi)) s = 0.5 * (lo + hi);
  if (!(s > lo && s < hi)) return KEP_ERR_CLUSTER;    // lo and hi are adjacent doubles
  *sigma = s;
  return KEP_OK;
}

extern "C" kep_status kep_interp_update(kep_interp_state* st, int64_t k, double sigma, int64_t nu) {
  if (!st || !interp_bracket_ok(st, k)) return KEP_ERR_INVALID;
  if (!(sigma > st->lo && sigma < st->hi) || nu < st->nu_lo || nu > st->nu_hi) return KEP_ERR_INVALID;
  const bool midpoint = st->bisect_next != 0;
  const double kd = static_cast<double>(k);
  if (nu >= k) {
    // the upper end moves; a lower end kept twice in a row is pulled halfway towards k
    if (st->last == 1 && !midpoint) st->w_lo = kd - 0.5 * (kd - st->w_lo);
    st->hi = sigma; st->nu_hi = nu; st->w_hi = static_cast<double>(nu);
    st->last = 1;
  } else {
    if (st->last == -1 && !midpoint) st->w_hi = kd + 0.5 * (st->w_hi - kd);
    st->lo = sigma; st->nu_lo = nu; st->w_lo = static_cast<double>(nu);
    st->last = -1;
  }
  const int64_t wnow = st->nu_hi - st->nu_lo;
  // keep the last four widths: the safeguard compares with the width three steps back
  if (st->nwidth == 4) {
    for (int i = 0; i < 3; ++i) st->width[i] = st->width[i + 1];
    st->width[3] = wnow;
  } else {
    st->width[st->nwidth++] = wnow;
  }
  st->bisect_next = (!midpoint && st->nwidth == 4 && 2 * wnow > st->width[0]) ? 1 : 0;
  return KEP_OK;
}

extern "C" kep_status kep_kth_eigenpair(kep_ctx* c, int64_t k, const kep_params* params, double* lambda,
                                        double* x_out, kep_report* report) {
  if (!c || !lambda) return KEP_ERR_INVALID;
  const int64_t n = c->plan.n;                        // vector length (2 herm_n for a Hermitian pencil)
  const int64_t n_eig = c->herm_n ? c->herm_n : n;    // eigenvalues counted by nu
  if (k < 1 || k > n_eig) return KEP_ERR_INVALID;
  kep_params prm;
  if (params) prm = *params; else kep_default_params(&prm);
  if (prm.m_max < 1 || prm.max_lanczos < 2 || prm.max_si < 1) return KEP_ERR_INVALID;
  if (prm.b_factor < KEP_BFACTOR_AUTO || prm.b_factor > KEP_BFACTOR_OWN) return KEP_ERR_INVALID;
  if (prm.split != KEP_SPLIT_BISECT && prm.split != KEP_SPLIT_INTERP) return KEP_ERR_INVALID;
  if (prm.split == KEP_SPLIT_INTERP && prm.nshift > 1) return KEP_ERR_INVALID;
  int64_t cap = std::min<int64_t>(n + 1, std::max(prm.max_lanczos, prm.max_si) + 2);
  Driver* d = static_cast<Driver*>(c->driver);
  if (!d || d->cap_cols < cap) {
    c->driver_release();
    d = new Driver();
    c->driver = d;
    d->nblocks = std::max(1, std::min<int>(c->num_sms * 4, static_cast<int>((n + 255) / 256)));
    // the Lanczos bases V and B V: the columns asked for, fewer (at least 64) when device memory is
    // short (the largest problems: 2 GB stay free for the work vectors and the solves' buffers);
    // the iterations then stop at the basis size
    const int64_t cap_min = std::min<int64_t>(cap, 64);
    {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const int64_t room = static_cast<int64_t>(free_b) - (2ll << 30);
        const int64_t fit = room > 0 ? room / (16 * n) : 0;
        cap = std::max(cap_min, std::min(cap, fit));
      } else {
        cudaGetLastError();
      }
    }
    while (true) {
      if (cudaMalloc(&d->V, sizeof(double) * n * cap) == cudaSuccess) {
        if (cudaMalloc(&d->BV, sizeof(double) * n * cap) == cudaSuccess) break;
        cudaFree(d->V);
      }
      d->V = d->BV = nullptr;
      cudaGetLastError();
      if (cap == cap_min) { c->driver_release(); return KEP_ERR_NOMEM; }
      cap = std::max(cap_min, cap * 3 / 4);
    }
    d->cap_cols = cap;
    if (cudaMalloc(&d->w, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&d->u, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&d->u2, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&d->coef, sizeof(double) * cap) != cudaSuccess ||
        cudaMalloc(&d->partial, sizeof(double) * std::max<int64_t>(4, cap) * d->nblocks) != cudaSuccess) {
      c->driver_release();
      return KEP_ERR_NOMEM;
    }
  }
  cap = std::min(cap, d->cap_cols);
  Run R;
  R.c = c; R.d = d; R.n = n; R.norm_a = c->plan.norm_a_inf;
  R.ops.n = n; R.ops.num_blocks = d->nblocks; R.ops.partial = d->partial; R.ops.stream = c->stream;
  R.ops.timer = &c->timer;
  R.opsh = R.ops;
  if (c->herm_n) R.opsh.n = c->herm_n;
  kep_report& rep = R.rep;
  // the report is written on every return from here on, the partial one of a failed run included
  struct ReportOut {
    kep_report* dst;
    const kep_report* src;
    ~ReportOut() { if (dst) *dst = *src; }
  } report_out{report, &rep};
  rep.cap_cols = cap;
  std::vector<double> h_start(2 * n), tmp;
  if (prm.start_vectors) std::memcpy(h_start.data(), prm.start_vectors, sizeof(double) * 2 * n);
  else { gaussian_vector(prm.seed, n, h_start.data()); gaussian_vector(prm.seed + 1, n, h_start.data() + n); }

  auto t0 = clock_::now();
  double lo = 0, hi = 0;
  int64_t nl = 0, nh = n_eig;
  double nrm = 0;
  std::vector<double> alpha, beta;
  if (prm.init == KEP_INIT_GERSHGORIN) {
    // ---------------- stage 1, variant: an interval holding the whole spectrum ----------------
    // Every eigenvalue is a Rayleigh quotient x^T A x / x^T B x; Gershgorin bounds of A and of B
    // (B's lower bound positive) bound it: lambda >= loA / (loA < 0 ? loB : hiB) and
    // lambda <= hiA / (hiA > 0 ? loB : hiB).  nu there is 0 and n without a factorization.
    const int nb = d->nblocks;
    KEP_LAUNCH(&c->timer, KC_VEC, c->stream,
               gershgorin_kernel<<<nb, 256, 0, c->stream>>>(n, c->d_rp, c->d_ci, c->d_a, c->d_b, d->partial));
    std::vector<double> g(4 * static_cast<size_t>(nb));
    CTRY(cudaMemcpyAsync(g.data(), d->partial, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, c->stream));
    CTRY(cudaStreamSynchronize(c->stream));
    double loA = INFINITY, hiA = -INFINITY, loB = INFINITY, hiB = -INFINITY;
    for (int q = 0; q < nb; ++q) {
      loA = std::min(loA, g[q]); hiA = std::max(hiA, g[nb + q]);
      loB = std::min(loB, g[2 * nb + q]); hiB = std::max(hiB, g[3 * nb + q]);
    }
    if (!(loB > 0.0)) return KEP_ERR_INVALID;          // B not shown positive definite by its discs
    lo = loA / (loA < 0 ? loB : hiB);
    hi = hiA / (hiA > 0 ? loB : hiB);
    const double pad = 1e-12 * std::max({std::fabs(lo), std::fabs(hi), 1.0});
    lo -= pad;
    hi += pad;
    nl = 0;
    nh = n_eig;
  } else {
  // ---------------- stage 1: Algorithm 2 ----------------
  DTRY(R.choose_bslot(prm.b_factor));
  DTRY(R.factor_B());
  CTRY(cudaMemcpyAsync(d->V, h_start.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  DTRY(R.b_normalize(0, nrm));                        // v_1 := v_1 / ||v_1||_B
  int64_t nu_prev = 0, nu_cur = 0;                    // nu^(0) := 0
  double sig_prev = 0, sig_cur = 0;
  bool bracketed = false;
  for (int64_t j = 1; j <= prm.max_lanczos && j < cap; ++j) {
    double* vj = R.col(d->V, j - 1);
    DTRY(ctx_spmv_dev(c, vj, d->u, nullptr));         // u = A v_j
    double a = 0;
    DTRY(R.dots(vj, 1, d->u, &a));                    // alpha_j = v_j^T A v_j
    DTRY(R.solve_B(d->u, d->w));                      // w = B^{-1} A v_j
    R.ops.axpby(-a, vj, 1.0, d->w);
    if (j > 1) R.ops.axpby(-beta.back(), R.col(d->V, j - 2), 1.0, d->w);
    DTRY(R.reorth(static_cast<int32_t>(j), d->w, tmp));
    CTRY(cudaMemcpyAsync(R.col(d->V, j), d->w, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    double b = 0;
    DTRY(R.b_normalize(j, b));                        // beta_j = ||w||_B, v_{j+1} = w / beta_j
    alpha.push_back(a);
    beta.push_back(b);
    // Ritz values of T_j (Eq. 2.3): the extreme ones are needed
    const int m = static_cast<int>(j);
    std::vector<double> wv(m), Z(static_cast<size_t>(m) * m);
    if (!tridiag_eigen(m, alpha.data(), beta.data(), wv.data(), Z.data())) return KEP_ERR_NOT_CONVERGED;
    sig_cur = (k <= nu_prev) ? wv[0] : wv[m - 1];
    DTRY(R.nu_at(sig_cur, nu_cur));
    rep.n_lanczos = j;
    if (j != 1 && ((nu_cur < k && k <= nu_prev) || (nu_prev < k && k <= nu_cur))) { bracketed = true; break; }
    nu_prev = nu_cur;
    sig_prev = sig_cur;
  }
  if (!bracketed) return KEP_ERR_NOT_CONVERGED;
  lo = std::min(sig_prev, sig_cur); hi = std::max(sig_prev, sig_cur);
  nl = std::min(nu_prev, nu_cur); nh = std::max(nu_prev, nu_cur);
  }
  rep.init_lo = lo; rep.init_hi = hi; rep.init_nu_lo = nl; rep.init_nu_hi = nh;
  rep.t_stage[0] = seconds_since(t0);

  // ---------------- stage 2: Algorithm 1' (bisection, or multisection with nshift points) ----------------
  t0 = clock_::now();
  const int32_t ns = std::max(1, prm.nshift);
  std::vector<double> sig(ns);
  std::vector<int64_t> nus(ns);
  if (prm.split == KEP_SPLIT_INTERP && nh - nl > prm.m_max) {
    kep_interp_state is;
    DTRY(kep_interp_init(k, lo, hi, nl, nh, &is));
    while (is.nu_hi - is.nu_lo > prm.m_max) {
      double s = 0;
      int64_t v = 0;
      DTRY(kep_interp_point(&is, k, prm.m_max, &s));
      DTRY(R.nu_at(s, v));
      DTRY(kep_interp_update(&is, k, s, v));
      rep.n_bisect++;
      if (rep.n_bisect > 200) return KEP_ERR_CLUSTER;
    }
    lo = is.lo; hi = is.hi; nl = is.nu_lo; nh = is.nu_hi;
  }
  while (nh - nl > prm.m_max) {
    // the shifts in increasing order; once one of them reaches k the later ones are not needed
    DTRY(kep_multisection_points(lo, hi, ns, sig.data()));
    int32_t used = 0;
    for (int32_t q = 0; q < ns; ++q) {
      DTRY(R.nu_at(sig[q], nus[q]));
      used = q + 1;
      if (k <= nus[q]) break;
    }
    DTRY(kep_multisection_update(k, used, sig.data(), nus.data(), &lo, &hi, &nl, &nh));
    rep.n_bisect++;
    if (rep.n_bisect > 200) return KEP_ERR_CLUSTER;    // a multiple eigenvalue can stall the count
  }
  rep.sigma_lo = lo; rep.sigma_hi = hi; rep.nu_lo = nl; rep.nu_hi = nh;
  rep.t_stage[1] = seconds_since(t0);

  // ---------------- stage 3: Algorithm 3 ----------------
  t0 = clock_::now();
  const int64_t l = k - nl, mm = nh - nl;
  double sigma = 0.5 * (lo + hi);
  const bool f32ir = prm.solve_precision == KEP_SOLVE_F32_IR;
  // v_1 = B^{-1} v~_1, so that ||v_1||_B = ||v~_1||_{B^{-1}} (formed before the shifted factor,
  // which may take B's slot)
  if (prm.init == KEP_INIT_GERSHGORIN) DTRY(R.choose_bslot(prm.b_factor));
  CTRY(cudaMemcpyAsync(d->u, h_start.data() + n, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  DTRY(R.solve_B(d->u, d->V));
  DTRY(R.b_normalize(0, nrm));
  {
    int64_t nu_mid = 0;
    const int mode = c->schur_mode;
    if (f32ir) c->schur_mode = KEP_SCHUR_FP32;         // reduced-precision factor, refined solves
    const kep_status fs = R.nu_at(sigma, nu_mid);     // factor of A - sigma B kept in slot 0
    c->schur_mode = mode;
    DTRY(fs);
  }
  // w = (A - sigma B)^{-1} rhs with the factor in slot 0 (refined when it is a reduced one)
  bool refine_all = f32ir;          // every solve refined (a reduced factor, or a restart)
  auto shifted_solve = [&](const double* rhs, double* out) -> kep_status {
    if (!refine_all) return ctx_solve_dev(c, 0, rhs, out);
    int32_t it = 0;
    double be = 0.0;
    const kep_status st = ctx_solve_refined_dev(c, rhs, out, 1e-13, 100, &it, &be);
    rep.n_refine += it;
    rep.solve_berr = std::max(rep.solve_berr, be);
    return st;
  };
  alpha.clear(); beta.clear();
  std::vector<double> G;                              // 2-norm Gram matrix of [v_1 .. v_{j+1}]
  int64_t gcap = cap;
  G.assign(static_cast<size_t>(gcap) * gcap, 0.0);
  {
    double g = 0;
    DTRY(R.dots(d->V, 1, d->V, &g));
    G[0] = g;
  }
  std::vector<double> prev_c;                         // coefficients of x^{(j-1)}_i, i <= m, in V
  int64_t prev_j = -1;
  bool converged = false;
  std::vector<double> res_lam, res_eta, best_coef;
  int64_t best_j = 0;
  for (int64_t j = 1; j <= prm.max_si && j + 1 < cap; ++j) {
    double* vj = R.col(d->V, j - 1);
    double* bvj = R.col(d->BV, j - 1);
    DTRY(shifted_solve(bvj, d->w));                   // w = (A - sigma B)^{-1} B v_j
    double a = 0;
    DTRY(R.dots(bvj, 1, d->w, &a));                   // alpha~_j = (B v_j)^T w
    R.ops.axpby(-a, vj, 1.0, d->w);
    if (j > 1) R.ops.axpby(-beta.back(), R.col(d->V, j - 2), 1.0, d->w);
    DTRY(R.reorth(static_cast<int32_t>(j), d->w, tmp));
    CTRY(cudaMemcpyAsync(R.col(d->V, j), d->w, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    double b = 0;
    DTRY(R.b_normalize(j, b));
    alpha.push_back(a);
    beta.push_back(b);
    {   // new column of the Gram matrix
      std::vector<double> gc(j + 1);
      DTRY(R.dots(d->V, static_cast<int32_t>(j + 1), R.col(d->V, j), gc.data()));
      for (int64_t i = 0; i <= j; ++i) { G[i * gcap + j] = gc[i]; G[j * gcap + i] = gc[i]; }
    }
    rep.n_si_iter = j;
    if (j < mm) continue;
    const int m = static_cast<int>(j);
    std::vector<double> th(m), Y(static_cast<size_t>(m) * m);
    if (!tridiag_eigen(m, alpha.data(), beta.data(), th.data(), Y.data())) return KEP_ERR_NOT_CONVERGED;
    // order by |theta~| descending (Eq. 3.2)
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int p1, int p2) { return std::fabs(th[p1]) > std::fabs(th[p2]); });
    const double bj = b;
    double bnext_2norm = std::sqrt(std::max(0.0, G[j * gcap + j]));   // ||v_{j+1}||_2
    // ||B v_{j+1}||_2 for the residual identity
    double bvn = 0;
    DTRY(R.dots(R.col(d->BV, j), 1, R.col(d->BV, j), &bvn));
    bvn = std::sqrt(bvn);
    (void)bnext_2norm;
    std::vector<double> lam_i(mm), eta_i(mm), rest(mm), coef(static_cast<size_t>(mm) * (j + 1));
    for (int64_t ii = 0; ii < mm; ++ii) {
      const int p = ord[ii];
      const double t = th[p];
      const double* y = Y.data() + static_cast<size_t>(p) * m;
      lam_i[ii] = sigma + 1.0 / t;                       // Eq. 2.7
      const double rho = std::fabs(bj * y[m - 1] / t);
      eta_i[ii] = (1.0 / std::fabs(t)) * rho / std::sqrt(1.0 + rho * rho);   // Eq. 3.1
      double* cc = coef.data() + ii * (j + 1);
      for (int q2 = 0; q2 < m; ++q2) cc[q2] = t * y[q2];   // x_{i,2} = theta V y + v_{j+1} beta (e_j^T y)
      cc[m] = bj * y[m - 1];
      double xn2 = 0;                                  // ||x||_2^2 = c^T G c
      for (int64_t r1 = 0; r1 <= j; ++r1) {
        double s = 0;
        for (int64_t r2 = 0; r2 <= j; ++r2) s += G[r1 * gcap + r2] * cc[r2];
        xn2 += cc[r1] * s;
      }
      rest[ii] = bvn * std::fabs(bj * y[m - 1] / t) / std::sqrt(std::max(xn2, 1e-300));   // Eq. 2.12
    }
    // inclusion (3.3) and disjointness (3.4)
    bool ok = true;
    for (int64_t ii = 0; ii < mm; ++ii)
      if (!(lam_i[ii] - eta_i[ii] >= lo && lam_i[ii] + eta_i[ii] < hi)) ok = false;
    std::vector<int> s_ord(mm);
    std::iota(s_ord.begin(), s_ord.end(), 0);
    std::sort(s_ord.begin(), s_ord.end(), [&](int p1, int p2) { return lam_i[p1] < lam_i[p2]; });
    for (int64_t ii = 0; ii + 1 < mm; ++ii)
      if (!(lam_i[s_ord[ii]] + eta_i[s_ord[ii]] < lam_i[s_ord[ii + 1]] - eta_i[s_ord[ii + 1]])) ok = false;
    if (ok && rep.si_iter_bound == 0) rep.si_iter_bound = j;
    for (int64_t ii = 0; ii < mm; ++ii) if (!(rest[ii] < prm.tau_res)) ok = false;
    rep.last_res = *std::max_element(rest.begin(), rest.end());
    // relative difference (Eq. 3.5) between iterations j-1 and j, through the Gram matrix
    bool diff_ok = prev_j == j - 1;
    rep.last_diff = -1.0;
    if (diff_ok) {
      for (int64_t ii = 0; ii < mm; ++ii) {
        const double* cn = coef.data() + ii * (j + 1);
        const double* co = prev_c.data() + ii * j;    // length j (basis v_1..v_j)
        std::vector<double> cpad(j + 1, 0.0), dv(j + 1);
        for (int64_t r = 0; r < j; ++r) cpad[r] = co[r];
        auto gram = [&](const double* u1, const double* u2) {
          double acc = 0;
          for (int64_t r1 = 0; r1 <= j; ++r1) {
            double s2 = 0;
            for (int64_t r2 = 0; r2 <= j; ++r2) s2 += G[r1 * gcap + r2] * u2[r2];
            acc += u1[r1] * s2;
          }
          return acc;
        };
        const double nn = gram(cn, cn), no = gram(cpad.data(), cpad.data()), dot = gram(cn, cpad.data());
        // scale x^{(j)} to the 2-norm of x^{(j-1)} with the sign that aligns them, then subtract
        // in coefficient space (no cancellation between large norms)
        const double s = (dot >= 0 ? 1.0 : -1.0) * std::sqrt(no / std::max(nn, 1e-300));
        for (int64_t r = 0; r <= j; ++r) dv[r] = s * cn[r] - cpad[r];
        const double dn2 = gram(dv.data(), dv.data());
        const double rd = std::sqrt(std::max(dn2, 0.0)) / std::sqrt(std::max(no, 1e-300));
        rep.last_diff = std::max(rep.last_diff, rd);
        if (!(rd < prm.tau_diff)) diff_ok = false;
      }
    }
    prev_c.assign(static_cast<size_t>(mm) * (j + 1), 0.0);
    for (int64_t ii = 0; ii < mm; ++ii)
      for (int64_t r = 0; r <= j; ++r) prev_c[ii * (j + 1) + r] = coef[ii * (j + 1) + r];
    // prev_c is read next iteration with stride j+1 == (next j)
    prev_j = j;
    if (!(ok && diff_ok)) continue;
    // confirm the residuals explicitly: ||(A - lambda B) x||_2 / ||x||_2 < tau_res for i <= m
    bool explicit_ok = true;
    rep.last_res_explicit = 0.0;
    for (int64_t ii = 0; ii < mm && explicit_ok; ++ii) {
      CTRY(cudaMemcpyAsync(d->coef, coef.data() + ii * (j + 1), sizeof(double) * (j + 1), cudaMemcpyHostToDevice,
                           c->stream));
      R.ops.combine(d->V, n, static_cast<int32_t>(j + 1), d->coef, 1.0, 0.0, d->w);
      DTRY(ctx_spmv_dev(c, d->w, d->u, d->u2));
      R.ops.resid_partials(d->u, d->u2, lam_i[ii], d->w);
      std::vector<double> part(2 * d->nblocks);
      DTRY(R.to_host(part.data(), d->partial, 2 * d->nblocks));
      double rr = 0, xx = 0;
      for (int bb = 0; bb < d->nblocks; ++bb) { rr += part[2 * bb]; xx += part[2 * bb + 1]; }
      const double rel = std::sqrt(rr) / std::sqrt(std::max(xx, 1e-300));
      rep.last_res_explicit = std::max(rep.last_res_explicit, rel);
      if (!(rel < prm.tau_res)) explicit_ok = false;
    }
    if (!explicit_ok && !refine_all) {
      // The Lanczos relation and the relative differences say the interval's pairs have converged,
      // but their explicit residuals stay above tau_res: the rounding of the shifted solves sets a
      // floor (the factor's backward error times ||A||), so the Ritz vectors are those of a pencil
      // perturbed by that much.  Algorithm 3 is run again, once, from the same start vector with
      // every shifted solve refined in FP64 (GMRES with the factor as preconditioner) to a backward
      // error of 1e-13.
      refine_all = true;
      rep.restarted = 1;
      alpha.clear(); beta.clear();
      const double g0 = G[0];
      std::fill(G.begin(), G.end(), 0.0);
      G[0] = g0;
      prev_c.clear();
      prev_j = -1;
      rep.si_iter_bound = 0;
      j = 0;
      continue;
    }
    if (!explicit_ok) continue;
    converged = true;
    // sort the interval's pairs increasingly and take the l-th (Algorithm 3, last two lines)
    const int64_t pick = s_ord[l - 1];
    best_coef.assign(coef.begin() + pick * (j + 1), coef.begin() + (pick + 1) * (j + 1));
    best_j = j;
    res_lam = lam_i; res_eta = eta_i;
    rep.lambda = lam_i[pick];
    rep.eta = eta_i[pick];
    break;
  }
  if (!converged) return KEP_ERR_CLUSTER;
  // x_k = V c, B-normalized; explicit residuals for the report
  CTRY(cudaMemcpyAsync(d->coef, best_coef.data(), sizeof(double) * (best_j + 1), cudaMemcpyHostToDevice, c->stream));
  R.ops.combine(d->V, n, static_cast<int32_t>(best_j + 1), d->coef, 1.0, 0.0, d->w);
  DTRY(ctx_spmv_dev(c, d->w, d->u, d->u2));
  double xbx = 0;
  DTRY(R.dots(d->w, 1, d->u2, &xbx));
  const double xs = 1.0 / std::sqrt(xbx);
  R.ops.axpby(0.0, d->w, xs, d->w);
  R.ops.axpby(0.0, d->u, xs, d->u);
  R.ops.axpby(0.0, d->u2, xs, d->u2);
  R.ops.resid_partials(d->u, d->u2, rep.lambda, d->w);
  {
    std::vector<double> part(2 * d->nblocks);
    DTRY(R.to_host(part.data(), d->partial, 2 * d->nblocks));
    double rr = 0, xx = 0;
    for (int bb = 0; bb < d->nblocks; ++bb) { rr += part[2 * bb]; xx += part[2 * bb + 1]; }
    rep.rel_res = std::sqrt(rr) / std::sqrt(xx);
    rep.rel_res_normwise = rep.rel_res / std::max(R.norm_a, 1e-300);
  }
  if (x_out) {
    if (c->herm_n) {                                   // [Re x; Im x] -> interleaved complex
      DTRY(herm_to_interleaved(c, d->w, d->u));
      DTRY(R.to_host(x_out, d->u, n));
    } else {
      DTRY(R.to_host(x_out, d->w, n));
    }
  }
  rep.t_stage[2] = seconds_since(t0);
  *lambda = rep.lambda;
  if (report) *report = rep;
  return KEP_OK;
}
