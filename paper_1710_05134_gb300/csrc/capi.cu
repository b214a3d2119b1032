// C ABI of the kep library: context lifecycle, symbolic analysis upload, factor, solve, SpMV.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kep_ctx.h"
#include "kep_vec.h"

static_assert(KEP_NKCLASS == kep::KC_COUNT, "kernel class count");

using namespace kep;

namespace kep {

template <typename T>
static kep_status dev_upload(kep_ctx* c, T** out, const std::vector<T>& v) {
  *out = nullptr;
  size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return KEP_ERR_NOMEM;
  c->allocs.push_back(p);
  if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return KEP_ERR_CUDA;
  *out = static_cast<T*>(p);
  return KEP_OK;
}

template <typename T>
static kep_status dev_alloc(kep_ctx* c, T** out, size_t count, bool plan_dependent = false) {
  *out = nullptr;
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();                  // an allocation failure is reported, not left pending
    return KEP_ERR_NOMEM;
  }
  (plan_dependent ? c->mem_allocs : c->allocs).push_back(p);
  *out = static_cast<T*>(p);
  return KEP_OK;
}

template <typename T>
static kep_status dev_upload_mem(kep_ctx* c, const T** out, const std::vector<T>& v) {
  T* p = nullptr;
  kep_status st = dev_alloc(c, &p, v.size(), true);
  if (st != KEP_OK) return st;
  if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return KEP_ERR_CUDA;
  *out = p;
  return KEP_OK;
}


static kep_status alloc_slot(kep_ctx* c, int i) {
  if (c->slot_ready[i]) return KEP_OK;
  const Plan& P = c->plan;
  FactorSlot& S = c->slot[i];
  KEP_TRY(dev_alloc(c, &S.F, P.front_total, true));
  KEP_TRY(dev_alloc(c, &S.rowvar, P.vec_total, true));
  KEP_TRY(dev_alloc(c, &S.apos, P.vec_total, true));
  KEP_TRY(dev_alloc(c, &S.Dd, P.piv_total, true));
  KEP_TRY(dev_alloc(c, &S.De, P.piv_total, true));
  KEP_TRY(dev_alloc(c, &S.piv, P.piv_total, true));
  KEP_TRY(dev_alloc(c, &S.d_in, P.nfronts, true));
  KEP_TRY(dev_alloc(c, &S.nelim, P.nfronts, true));
  KEP_TRY(dev_alloc(c, &S.d_out, P.nfronts, true));
  KEP_TRY(dev_alloc(c, &S.cnt, 3 * static_cast<size_t>(P.nfronts), true));
  KEP_TRY(dev_alloc(c, &S.status, 2, true));
  S.valid = false;
  c->slot_ready[i] = true;
  return KEP_OK;
}

// Upload the slack-dependent tables and allocate the slack-dependent workspaces.
kep_status setup_memory(kep_ctx* c) {
  const Plan& P = c->plan;
  KEP_TRY(dev_upload_mem(c, &c->T.m_alloc, P.m_alloc));
  KEP_TRY(dev_upload_mem(c, &c->T.front_off, P.front_off));
  KEP_TRY(dev_upload_mem(c, &c->T.vec_off, P.vec_off));
  KEP_TRY(dev_upload_mem(c, &c->T.piv_off, P.piv_off));
  const int64_t* p21 = nullptr;
  KEP_TRY(dev_upload_mem(c, &p21, P.p21_off));
  c->W.p21_off = const_cast<int64_t*>(p21);
  KEP_TRY(dev_alloc(c, &c->W.P21, std::max<int64_t>(P.max_large_rows, 1) * kPanel, true));
  KEP_TRY(dev_alloc(c, &c->d_vasm, P.vec_total, true));
  KEP_TRY(dev_alloc(c, &c->d_vfac, P.vec_total, true));
  std::vector<int32_t> fbase;
  const int64_t nflags = df_flag_bases(P, fbase);
  KEP_TRY(dev_alloc(c, &c->d_df_flags, nflags, true));
  if (cudaMemset(c->d_df_flags, 0, sizeof(int32_t) * std::max<int64_t>(nflags, 1)) != cudaSuccess) return KEP_ERR_CUDA;
  KEP_TRY(dev_alloc(c, &c->d_df_pcnt, nflags, true));
  c->df_nflags = nflags;
  for (int i = 0; i < 2; ++i) KEP_TRY(dev_alloc(c, &c->d_df_part_base[i], P.nfronts, true));
  const int32_t* fb = nullptr;
  KEP_TRY(dev_upload_mem(c, &fb, fbase));
  c->d_df_fbase = const_cast<int32_t*>(fb);
  return KEP_OK;
}

void release_memory(kep_ctx* c) {
  cudaStreamSynchronize(c->stream);
  c->graphs.clear();                     // they hold pointers into the storage freed here
  for (void* p : c->mem_allocs) cudaFree(p);
  c->mem_allocs.clear();
  c->emul_ws = nullptr;
  c->emul_bytes = 0;
  for (auto& ep : c->emul_plan) { ep.min_planned = -1; ep.G = 0; ep.d_off = nullptr; ep.h_end.clear(); }
  for (int i = 0; i < 2; ++i) {
    c->slot_ready[i] = false;
    c->slot[i].valid = false;
    c->d_df_items[i] = nullptr;
    c->df_items_cap[i] = 0;
    c->df_version[i] = 0;
  }
  c->d_df_flags = nullptr;
  c->d_df_fbase = nullptr;
  c->d_df_pcnt = nullptr;
  c->d_df_part_base[0] = c->d_df_part_base[1] = nullptr;
  c->d_df_part = nullptr;
  c->df_part_cap = 0;
  c->multi_cap = 0;
  c->ent_G = 0;
  c->d_ent_front = nullptr;
  c->d_ent_shift = nullptr;
  {   // entry arrays grown for a multisection step were plan-dependent: back to the originals
    const double* p21 = c->W.P21;
    const int64_t* p21o = c->W.p21_off;
    c->W = c->W0;
    c->W.P21 = const_cast<double*>(p21);
    c->W.p21_off = const_cast<int64_t*>(p21o);
    c->w_cap_entries = c->W0.cap;
  }
}

// Delayed pivots overflowed the slack of some fronts of the given factorizations: grow those
// fronts' slack to what they had to hold (plus a quarter and 16), or, when no front recorded a
// size, every non-leaf front's slack twofold; then rebuild the slack-dependent storage (the
// ordering, tree and index maps stay).  Only the fronts that overflowed grow, so the storage of the
// largest problems stays within the device.
static kep_status replan(kep_ctx* c, const std::vector<const FactorSlot*>& failed) {
  Plan& P = c->plan;
  std::vector<int32_t> din(P.nfronts);
  bool grew = false;
  for (const FactorSlot* S : failed) {
    if (cudaMemcpy(din.data(), S->d_in, sizeof(int32_t) * P.nfronts, cudaMemcpyDeviceToHost) != cudaSuccess)
      return KEP_ERR_CUDA;
    for (int32_t t = 0; t < P.nfronts; ++t)
      if (din[t] < -1) {
        const int64_t need = -static_cast<int64_t>(din[t]) - 1;
        const int32_t ns = static_cast<int32_t>(need + need / 4 + 16);
        if (ns > P.slack[t]) { P.slack[t] = ns; grew = true; }
      }
  }
  if (!grew)
    for (int32_t t = 0; t < P.nfronts; ++t)
      if (P.child_ptr[t + 1] != P.child_ptr[t]) P.slack[t] = std::max(2 * P.slack[t], 16);
  release_memory(c);
  layout_memory(P);
  ++c->replans;
  return setup_memory(c);
}

// Counts of a Hermitian pencil from those of its real embedding, which has every eigenvalue
// twice: half of each.  An odd count means an eigenvalue within rounding of the shift (the pair's
// two copies fell on both sides), reported like an exact zero pivot.
static kep_status herm_counts(kep_ctx* c, kep_status st, kep_inertia* out) {
  if (!c->herm_n || !out || (st != KEP_OK && st != KEP_ERR_SINGULAR)) return st;
  const bool odd = (out->neg & 1) || (out->pos & 1);
  out->neg /= 2;
  out->pos /= 2;
  out->zero = c->herm_n - out->neg - out->pos;
  return (odd || out->zero > 0) ? KEP_ERR_SINGULAR : st;
}

// Tensor-core batches for G shifts: a level's entries on the tensor-core path (consecutive in its
// front-major entry list, at most emul_max_batch() entries and kEmulBudget bytes of workspace
// each) and each entry's workspace offset inside its batch.
static kep_status plan_emul(kep_ctx* c, int G, int64_t min_front, kep_ctx::EmulPlan*& out) {
  out = nullptr;
  kep_ctx::EmulPlan& ep = c->emul_plan[G == 1 ? 0 : 1];
  if (ep.min_planned != min_front || ep.G != G) {
    const Plan& P = c->plan;
    constexpr int64_t kEmulBudget = 24ll << 30;
    const int64_t nent = static_cast<int64_t>(P.nfronts) * G;
    std::vector<int64_t> off(nent, 0);
    ep.h_end.assign(nent, 0);
    int64_t need = 0;
    for (int32_t l = 0; l < P.nlevels; ++l) {
      const int32_t lb = P.level_ptr[l] * G, le = P.level_ptr[l + 1] * G;
      auto front = [&](int32_t e) { return P.level_fronts[P.level_ptr[l] + (e - lb) / G]; };
      int32_t e = lb;
      while (e < le) {
        if (P.m_alloc[front(e)] < min_front) { ++e; continue; }
        const int32_t start = e;
        int64_t bytes = 0;
        while (e < le && P.m_alloc[front(e)] >= min_front && e - start < emul_max_batch()) {
          const int64_t fb = (static_cast<int64_t>(emul_workspace_bytes(P.m_alloc[front(e)])) + 255) / 256 * 256;
          if (e > start && bytes + fb > kEmulBudget) break;
          off[e] = bytes;
          bytes += fb;
          ++e;
        }
        ep.h_end[start] = e - lb;
        need = std::max(need, bytes);
      }
    }
    if (need > c->emul_bytes) {
      void* p = nullptr;
      if (cudaMalloc(&p, need) != cudaSuccess) { cudaGetLastError(); return KEP_ERR_NOMEM; }
      if (cudaMemset(p, 0, need) != cudaSuccess) return KEP_ERR_CUDA;
      c->mem_allocs.push_back(p);
      c->emul_ws = p;
      c->emul_bytes = need;
    }
    if (!ep.d_off) {   // capacity for the largest G this plan can serve
      int64_t* p = nullptr;
      KEP_TRY(dev_alloc(c, &p, static_cast<int64_t>(P.nfronts) * (G == 1 ? 1 : kMaxShifts), true));
      ep.d_off = p;
    }
    if (cudaMemcpy(ep.d_off, off.data(), sizeof(int64_t) * nent, cudaMemcpyHostToDevice) != cudaSuccess)
      return KEP_ERR_CUDA;
    ep.G = G;
    ep.min_planned = need > 0 ? min_front : -2;
  }
  if (c->emul_bytes > 0 && ep.min_planned == min_front) out = &ep;
  return KEP_OK;
}

// Factor the G matrices ca[g] A + cb[g] B in the same launches; shift g's factor goes to slots[g]
// with contribution-block pool pools[g] and L21 workspace p21[g].
static kep_status factor_set(kep_ctx* c, int G, FactorSlot* const* slots, double* const* pools,
                             double* const* p21, const double* ca, const double* cb, kep_inertia* out, int* bits) {
  const Plan& P = c->plan;
  FactorLaunch F;
  F.plan = &P;
  F.T = c->T;
  F.SS.n = G;
  for (int g = 0; g < G; ++g) {
    slots[g]->valid = false;
    F.SS.s[g] = *slots[g];
    F.SS.cbpool[g] = pools[g];
    F.SS.P21[g] = p21[g];
  }
  F.G = G;
  if (G == 1) {
    F.W = c->W;
    F.d_ent_front = c->d_level_fronts;
    F.d_ent_shift = nullptr;
    F.h_ent_front = P.level_fronts.data();
  } else {
    F.W = c->W;               // the entry arrays of c->W were grown to level width x G
    F.d_ent_front = c->d_ent_front;
    F.d_ent_shift = c->d_ent_shift;
    F.h_ent_front = c->h_ent_front.data();
  }
  F.h_done = c->h_done;
  F.d_red = c->d_red;
  F.h_red = c->h_red;
  F.stream = c->stream;
  F.num_sms = c->num_sms;
  F.timer = &c->timer;
  F.flops = c->d_flops;
  F.graphs = &c->graphs;
  if (!c->capture_stream && cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->capture_stream = nullptr;
  }
  F.capture_stream = c->capture_stream;
  // the tensor-core update for fronts of order >= emul_min_front: FP64-accurate (8 digits), or
  // the reduced-precision factor's 4 digits; smaller fronts FP64 or FP32 FMA tiles
  F.emul_min = c->schur_mode == KEP_SCHUR_FP64 ? 0 : c->emul_min_front;
  F.fp32_schur = c->schur_mode == KEP_SCHUR_FP32;
  F.schur_tile = c->schur_tile;
  F.emul_ws = nullptr;
  F.d_emul_off = nullptr;
  F.h_emul_end = nullptr;
  if (F.emul_min > 0) {
    kep_ctx::EmulPlan* ep = nullptr;
    KEP_TRY(plan_emul(c, G, F.emul_min, ep));
    if (ep) {
      F.emul_ws = c->emul_ws;
      F.d_emul_off = ep->d_off;
      F.h_emul_end = ep->h_end.data();
    } else {
      F.emul_min = 0;
    }
  }
  const kep_status st = run_factor(F, ca, cb, out, bits);
  if (st != KEP_OK) return st;
  for (int g = 0; g < G; ++g) { slots[g]->ca = ca[g]; slots[g]->cb = cb[g]; }
  return KEP_OK;
}

// Status of one factorization from its counts and bits; marks the slot valid when usable.
static kep_status finish_slot(kep_ctx* c, FactorSlot& S, const kep_inertia& in, int bits) {
  if (bits & ST_POOL) return KEP_ERR_POOL;
  if (bits & ST_NONFINITE) return KEP_ERR_NONFINITE;
  if (bits & ST_TIMEOUT) return KEP_ERR_TIMEOUT;
  if (in.neg + in.zero + in.pos != c->plan.n) return KEP_ERR_POOL;
  S.valid = true;
  return in.zero > 0 ? KEP_ERR_SINGULAR : KEP_OK;
}

// Host copies of a public slot's per-front counts (for the solves), after a factorization.
static kep_status record_slot(kep_ctx* c, int slot, int bits) {
  FactorSlot& S = c->slot[slot];
  c->slot_status[slot] = bits;
  c->slot_nelim[slot].resize(c->plan.nfronts);
  c->slot_din[slot].resize(c->plan.nfronts);
  if (cudaMemcpy(c->slot_nelim[slot].data(), S.nelim, sizeof(int32_t) * c->plan.nfronts,
                 cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(c->slot_din[slot].data(), S.d_in, sizeof(int32_t) * c->plan.nfronts,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return KEP_ERR_CUDA;
  ++c->factor_version[slot];
  return KEP_OK;
}

kep_status ctx_factor_once(kep_ctx* c, int slot, double ca, double cb, kep_inertia* out, int* bits_out) {
  FactorSlot* sp = &c->slot[slot];
  double* pool = c->d_cbpool;
  double* p21 = c->W.P21;
  kep_inertia in{0, 0, 0, 0};
  int bits = 0;
  const kep_status st = factor_set(c, 1, &sp, &pool, &p21, &ca, &cb, &in, &bits);
  *bits_out = bits;
  if (st != KEP_OK) return st;
  KEP_TRY(record_slot(c, slot, bits));
  if (out) *out = in;
  const kep_status fs = finish_slot(c, c->slot[slot], in, bits);
  c->slot_zero[slot] = c->slot[slot].valid ? in.zero : 0;
  return fs;
}

kep_status ctx_factor(kep_ctx* c, int slot, double ca, double cb, kep_inertia* out) {
  for (int attempt = 0;; ++attempt) {
    KEP_TRY(alloc_slot(c, slot));
    int bits = 0;
    kep_status st = ctx_factor_once(c, slot, ca, cb, out, &bits);
    if (st == KEP_ERR_POOL && (bits & ST_POOL) && attempt < 8) {
      KEP_TRY(replan(c, {&c->slot[slot]}));
      continue;
    }
    return herm_counts(c, st, out);
  }
}

// Device bytes one more shift of a multisection step needs: its slot, pool and L21 workspace.
static int64_t shift_bytes(const Plan& P) {
  return 8 * P.front_total + 8 * P.vec_total + 17 * P.piv_total + 24ll * P.nfronts + 8 * P.cb_total +
         8ll * std::max<int64_t>(P.max_large_rows, 1) * kPanel;
}

// Resources for G shifts in one launch sequence: G - 1 extra slots, pools and L21 workspaces,
// the front-major entry lists, and LargeWork entry arrays for level width x G.
static kep_status ensure_multi(kep_ctx* c, int G) {
  const Plan& P = c->plan;
  if (c->multi_cap < G) {
    for (int j = std::max(0, c->multi_cap - 1); j < G - 1; ++j) {
      FactorSlot& S = c->mslot[j];
      KEP_TRY(dev_alloc(c, &S.F, P.front_total, true));
      KEP_TRY(dev_alloc(c, &S.rowvar, P.vec_total, true));
      KEP_TRY(dev_alloc(c, &S.apos, P.vec_total, true));
      KEP_TRY(dev_alloc(c, &S.Dd, P.piv_total, true));
      KEP_TRY(dev_alloc(c, &S.De, P.piv_total, true));
      KEP_TRY(dev_alloc(c, &S.piv, P.piv_total, true));
      KEP_TRY(dev_alloc(c, &S.d_in, P.nfronts, true));
      KEP_TRY(dev_alloc(c, &S.nelim, P.nfronts, true));
      KEP_TRY(dev_alloc(c, &S.d_out, P.nfronts, true));
      KEP_TRY(dev_alloc(c, &S.cnt, 3 * static_cast<size_t>(P.nfronts), true));
      KEP_TRY(dev_alloc(c, &S.status, 2, true));
      KEP_TRY(dev_alloc(c, &c->mpool[j], P.cb_total, true));
      KEP_TRY(dev_alloc(c, &c->mp21[j], std::max<int64_t>(P.max_large_rows, 1) * kPanel, true));
      S.valid = false;
    }
    c->multi_cap = G;
  }
  if (c->ent_G != G) {
    const int64_t nent = static_cast<int64_t>(P.nfronts) * G;
    c->h_ent_front.resize(nent);
    std::vector<int8_t> sh(nent);
    for (int32_t q = 0; q < P.nfronts; ++q)       // level order kept: entry q G + g is front q, shift g
      for (int g = 0; g < G; ++g) {
        c->h_ent_front[static_cast<int64_t>(q) * G + g] = P.level_fronts[q];
        sh[static_cast<int64_t>(q) * G + g] = static_cast<int8_t>(g);
      }
    if (!c->d_ent_front) {   // capacity for kMaxShifts
      KEP_TRY(dev_alloc(c, &c->d_ent_front, static_cast<int64_t>(P.nfronts) * kMaxShifts, true));
      KEP_TRY(dev_alloc(c, &c->d_ent_shift, static_cast<int64_t>(P.nfronts) * kMaxShifts, true));
    }
    if (cudaMemcpy(c->d_ent_front, c->h_ent_front.data(), sizeof(int32_t) * nent, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_ent_shift, sh.data(), nent, cudaMemcpyHostToDevice) != cudaSuccess)
      return KEP_ERR_CUDA;
    c->ent_G = G;
  }
  const int32_t need = std::max<int32_t>(P.max_level_width, 1) * G;
  if (c->w_cap_entries < need) {
    LargeWork& W = c->W;
    KEP_TRY(dev_alloc(c, &W.k, need, true)); KEP_TRY(dev_alloc(c, &W.w, need, true));
    KEP_TRY(dev_alloc(c, &W.q, need, true)); KEP_TRY(dev_alloc(c, &W.fails, need, true));
    KEP_TRY(dev_alloc(c, &W.swap, need, true)); KEP_TRY(dev_alloc(c, &W.done, need, true));
    KEP_TRY(dev_alloc(c, &W.ws, need, true)); KEP_TRY(dev_alloc(c, &W.we, need, true));
    KEP_TRY(dev_alloc(c, &W.kend, need, true)); KEP_TRY(dev_alloc(c, &W.flush, need, true));
    KEP_TRY(dev_alloc(c, &W.reset, need, true)); KEP_TRY(dev_alloc(c, &W.finish, need, true));
    KEP_TRY(dev_alloc(c, &W.L11, static_cast<size_t>(need) * kPanel * kPanel, true));
    KEP_TRY(dev_alloc(c, &W.Dblk, static_cast<size_t>(need) * 2 * kPanel, true));
    KEP_TRY(dev_alloc(c, &W.pi, static_cast<size_t>(need) * kPanel, true));
    KEP_TRY(dev_alloc(c, &W.pt, static_cast<size_t>(need) * kPanel, true));
    KEP_TRY(dev_alloc(c, &W.colmax, static_cast<size_t>(need) * kPanel, true));
    int32_t* hd = nullptr;
    if (cudaMallocHost(reinterpret_cast<void**>(&hd), sizeof(int32_t) * need) != cudaSuccess) return KEP_ERR_NOMEM;
    if (c->h_done) cudaFreeHost(c->h_done);
    c->h_done = hd;
    W.cap = need;
    c->w_cap_entries = need;
  }
  return KEP_OK;
}

// Shifts one launch sequence can serve: at most kMaxShifts, as many as fit in free device memory
// (with 4 GB to spare).
static int multi_group(kep_ctx* c, int32_t ns) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); return 1; }
  const int64_t per = shift_bytes(c->plan);
  int have = std::max(1, c->multi_cap);
  int64_t avail = static_cast<int64_t>(free_b) - (4ll << 30);
  int G = have;
  while (G < std::min<int32_t>(ns, kMaxShifts) && avail >= per) { ++G; avail -= per; }
  return std::max(1, std::min<int>(G, std::min<int32_t>(ns, kMaxShifts)));
}

kep_status ctx_solve_dev(kep_ctx* c, int slot, const double* b, double* x) {
  FactorSlot& S = c->slot[slot];
  if (!c->slot_ready[slot] || !S.valid) return KEP_ERR_INVALID;
  if (c->slot_zero[slot] > 0) return KEP_ERR_SINGULAR;
  SolveLaunch L;
  L.plan = &c->plan;
  L.T = c->T;
  L.S = S;
  L.d_level_fronts = c->d_level_fronts;
  L.d_perm = c->d_perm;
  L.vasm = c->d_vasm;
  L.vfac = c->d_vfac;
  L.bnew = c->d_bnew;
  L.xnew = c->d_xnew;
  L.partial = c->d_solve_partial;
  L.h_nelim = c->slot_nelim[slot].data();
  if (c->df_version[slot] != c->factor_version[slot]) {
    // work items of the dataflow solve for this factorization (its delays and pivot counts)
    int64_t part_total = 0;
    build_df_items(c->plan, c->slot_nelim[slot].data(), c->slot_din[slot].data(), c->df_items[slot],
                   c->df_fwd_off[slot], c->df_bwd_off[slot], c->df_bwd_start[slot], c->df_part_base[slot],
                   part_total);
    if (part_total > c->df_part_cap) {
      double* pp = nullptr;
      KEP_TRY(dev_alloc(c, &pp, part_total + part_total / 4, true));
      c->d_df_part = pp;
      c->df_part_cap = part_total + part_total / 4;
    }
    if (cudaMemcpyAsync(c->d_df_part_base[slot], c->df_part_base[slot].data(), sizeof(int64_t) * c->plan.nfronts,
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    const int64_t need = std::max<int64_t>(1, static_cast<int64_t>(c->df_items[slot].size()));
    if (need > c->df_items_cap[slot]) {
      int2* p = nullptr;
      KEP_TRY(dev_alloc(c, &p, need + need / 4, true));
      c->d_df_items[slot] = p;
      c->df_items_cap[slot] = need + need / 4;
    }
    if (!c->df_items[slot].empty() &&
        cudaMemcpyAsync(c->d_df_items[slot], c->df_items[slot].data(), sizeof(int2) * c->df_items[slot].size(),
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    c->df_version[slot] = c->factor_version[slot];
  }
  L.df_fwd_items = c->d_df_items[slot];
  L.df_bwd_items = c->d_df_items[slot] + c->df_bwd_start[slot];
  L.h_df_fwd_off = c->df_fwd_off[slot].data();
  L.h_df_bwd_off = c->df_bwd_off[slot].data();
  L.df_counters = c->d_df_ctr;
  L.df_flags = c->d_df_flags;
  L.df_fbase = c->d_df_fbase;
  L.epoch = ++c->df_epoch;
  L.df_part = c->d_df_part;
  L.df_part_base = c->d_df_part_base[slot];
  L.df_pcnt = c->d_df_pcnt;
  L.df_nflags = c->df_nflags;
  L.stream = c->stream;
  L.num_sms = c->num_sms;
  L.timer = &c->timer;
  KEP_TRY(run_solve(L, b, x));
  // the dataflow kernels' bounded waits report through the first counter
  if (cudaMemcpyAsync(c->h_df_err, c->d_df_ctr, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return KEP_ERR_CUDA;
  return *c->h_df_err ? KEP_ERR_TIMEOUT : KEP_OK;
}

kep_status ctx_spmv_dev(kep_ctx* c, const double* x, double* ax, double* bx) {
  return run_spmv(c->plan.n, c->d_rp, c->d_ci, c->d_a, c->d_b, x, ax, bx, c->stream, c->num_sms, &c->timer);
}

}  // namespace kep

extern "C" {

void kep_default_params(kep_params* p) {
  if (!p) return;
  p->m_max = 20;
  p->tau_res = 1e-10;
  p->tau_diff = 1e-10;
  p->max_lanczos = 200;
  p->max_si = 300;
  p->start_vectors = nullptr;
  p->seed = 0x5eed;
  p->init = KEP_INIT_LANCZOS;
  p->nshift = 1;
  p->solve_precision = KEP_SOLVE_F64;
  p->b_factor = KEP_BFACTOR_AUTO;
  p->split = KEP_SPLIT_BISECT;
}

const char* kep_status_str(kep_status s) {
  switch (s) {
    case KEP_OK: return "ok";
    case KEP_ERR_INVALID: return "invalid argument or state";
    case KEP_ERR_NOT_SPD: return "B is not positive definite";
    case KEP_ERR_SINGULAR: return "exact zero pivot (shift is an eigenvalue)";
    case KEP_ERR_NOT_CONVERGED: return "iteration limit reached";
    case KEP_ERR_CLUSTER: return "interval eigenpairs could not be validated (cluster)";
    case KEP_ERR_POOL: return "delayed pivots exceeded the front slack";
    case KEP_ERR_TIMEOUT: return "device wait timed out";
    case KEP_ERR_CUDA: return "CUDA runtime error";
    case KEP_ERR_NONFINITE: return "non-finite pivot";
    case KEP_ERR_NOMEM: return "out of memory";
  }
  return "unknown status";
}

}  // extern "C"

namespace {
// The caller's pattern as a full symmetric CSR with sorted rows (values of A and B carried along;
// zeros when a_val / b_val are null), the caller entry of each position (src) and each caller
// entry's position (in2csr; bit 62 marks a lower off-diagonal entry standing for both triangles).
struct FullPattern {
  std::vector<int64_t> cnt, src, in2csr;
  std::vector<int32_t> ci;
  std::vector<double> av, bv;
};

kep_status full_pattern(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* a_val,
                        const double* b_val, bool lower, FullPattern& F) {
  if (n < 1 || n > INT32_MAX - 1 || !rowptr || !colind) return KEP_ERR_INVALID;
  if (rowptr[0] != 0) return KEP_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return KEP_ERR_INVALID;
  const int64_t nnz_in = rowptr[n];
  std::vector<int64_t>& cnt = F.cnt;
  cnt.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int64_t j = colind[e];
      if (j < 0 || j >= n) return KEP_ERR_INVALID;
      if (lower) {
        if (j > i) return KEP_ERR_INVALID;
        cnt[i + 1]++;
        if (j != i) cnt[j + 1]++;
      } else {
        cnt[i + 1]++;
      }
    }
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  const int64_t nnz = cnt[n];
  std::vector<int32_t>& ci = F.ci;
  std::vector<double>& av = F.av;
  std::vector<double>& bv = F.bv;
  std::vector<int64_t>& src = F.src;
  std::vector<int64_t>& in2csr = F.in2csr;
  ci.assign(nnz, 0); av.assign(nnz, 0.0); bv.assign(nnz, 0.0); src.assign(nnz, 0); in2csr.assign(nnz_in, 0);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int64_t j = colind[e];
        int64_t o = fill[i]++;
        const double a = a_val ? a_val[e] : 0.0, b = b_val ? b_val[e] : 0.0;
        ci[o] = static_cast<int32_t>(j); av[o] = a; bv[o] = b; src[o] = e;
        in2csr[e] = o;
        if (lower && j != i) {
          int64_t o2 = fill[j]++;
          ci[o2] = static_cast<int32_t>(i); av[o2] = a; bv[o2] = b; src[o2] = e;
        }
      }
  }
  std::vector<int64_t> idx;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t e0 = cnt[i], e1 = cnt[i + 1];
    bool sorted = true;
    for (int64_t e = e0 + 1; e < e1; ++e) if (ci[e] <= ci[e - 1]) { sorted = false; break; }
    if (sorted) continue;
    idx.resize(e1 - e0);
    for (int64_t e = e0; e < e1; ++e) idx[e - e0] = e;
    std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return ci[x] < ci[y]; });
    std::vector<int32_t> c2(e1 - e0); std::vector<double> a2(e1 - e0), b2(e1 - e0);
    std::vector<int64_t> s2(e1 - e0);
    for (int64_t k = 0; k < e1 - e0; ++k) {
      c2[k] = ci[idx[k]]; a2[k] = av[idx[k]]; b2[k] = bv[idx[k]]; s2[k] = src[idx[k]];
    }
    for (int64_t k = 0; k < e1 - e0; ++k) {
      ci[e0 + k] = c2[k]; av[e0 + k] = a2[k]; bv[e0 + k] = b2[k]; src[e0 + k] = s2[k];
    }
    for (int64_t e = e0 + 1; e < e1; ++e) if (ci[e] == ci[e - 1]) return KEP_ERR_INVALID;
  }
  {
    // the caller's entries' final positions: the slot in the entry's own row (the mirrored slot
    // of a lower off-diagonal entry carries the same value)
    std::vector<int64_t> rowof(nnz_in);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) rowof[e] = i;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) {
        const int64_t e = src[p];
        if (rowof[e] == i) in2csr[e] = p | ((lower && colind[e] != i) ? (1ll << 62) : 0ll);
      }
  }
  return KEP_OK;
}
}  // namespace

extern "C" {

kep_status kep_analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* a_val,
                       const double* b_val, int flags, const double* coords, kep_ctx** out) {
  if (!out) return KEP_ERR_INVALID;
  *out = nullptr;
  if (!a_val || !b_val) return KEP_ERR_INVALID;
  const bool lower = flags & KEP_PATTERN_LOWER;
  FullPattern FP;
  {
    const kep_status ps = full_pattern(n, rowptr, colind, a_val, b_val, lower, FP);
    if (ps != KEP_OK) return ps;
  }
  const int64_t nnz_in = rowptr[n];
  std::vector<int64_t>& cnt = FP.cnt;
  std::vector<int32_t>& ci = FP.ci;
  std::vector<double>& av = FP.av;
  std::vector<double>& bv = FP.bv;
  std::vector<int64_t>& src = FP.src;
  std::vector<int64_t>& in2csr = FP.in2csr;
  kep_ctx* c = new (std::nothrow) kep_ctx();
  if (!c) return KEP_ERR_NOMEM;
  for (int64_t i = 0; i < n; ++i) {
    double r = 0.0;
    for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) r += std::fabs(bv[p]);
    c->norm_b_inf = std::max(c->norm_b_inf, r);
  }
  c->nnz_in = nnz_in;
  c->lower_in = lower;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return KEP_ERR_CUDA; }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  std::string err;
  kep_status st = build_plan(n, cnt, ci, av, bv, coords, (flags & KEP_ORDER_GRAPH) != 0, (flags & KEP_ORDER_REFINED) != 0,
                             (flags & kOrderPairs) != 0, 8, c->plan, err);
  if (st != KEP_OK) { delete c; return st; }
  const Plan& P = c->plan;
#define UP(dst, vec) do { st = dev_upload(c, &dst, vec); if (st != KEP_OK) { kep_destroy(c); return st; } } while (0)
  int32_t *first, *p_sym, *m_sym, *parent, *child_ptr, *child_idx, *struct_var, *relmap, *ent_r, *ent_c;
  int64_t *struct_ptr, *relmap_ptr, *ent_ptr, *cb_off;
  double *ent_a, *ent_b;
  UP(first, P.first); UP(p_sym, P.p_sym); UP(m_sym, P.m_sym);
  UP(parent, P.parent); UP(child_ptr, P.child_ptr); UP(child_idx, P.child_idx);
  UP(struct_ptr, P.struct_ptr); UP(struct_var, P.struct_var);
  UP(relmap_ptr, P.relmap_ptr); UP(relmap, P.relmap);
  UP(ent_ptr, P.ent_ptr); UP(ent_r, P.ent_r); UP(ent_c, P.ent_c); UP(ent_a, P.ent_a); UP(ent_b, P.ent_b);
  UP(cb_off, P.cb_off);
  UP(c->d_level_fronts, P.level_fronts);
  UP(c->d_perm, P.perm);
  UP(c->d_iperm, P.iperm);
  UP(c->d_rp, cnt); UP(c->d_ci, ci); UP(c->d_a, av); UP(c->d_b, bv);
  UP(c->d_in2csr, in2csr);
#undef UP
  c->csr_src = std::move(src);
  FrontTables& T = c->T;
  T.nfronts = P.nfronts;
  T.first = first; T.p_sym = p_sym; T.m_sym = m_sym; T.parent = parent;
  T.child_ptr = child_ptr; T.child_idx = child_idx; T.struct_ptr = struct_ptr; T.struct_var = struct_var;
  T.relmap_ptr = relmap_ptr; T.relmap = relmap; T.ent_ptr = ent_ptr; T.ent_r = ent_r; T.ent_c = ent_c;
  T.ent_a = ent_a; T.ent_b = ent_b; T.cb_off = cb_off;
  // workspaces
  const int64_t ent = std::max<int32_t>(P.max_level_width, 1);
  LargeWork& W = c->W;
  W.cap = static_cast<int32_t>(ent);
  W.list = nullptr;
#define AL(dst, count) do { st = dev_alloc(c, &dst, count); if (st != KEP_OK) { kep_destroy(c); return st; } } while (0)
  AL(W.k, ent); AL(W.w, ent); AL(W.q, ent); AL(W.fails, ent); AL(W.swap, ent); AL(W.done, ent);
  AL(W.ws, ent); AL(W.we, ent); AL(W.kend, ent); AL(W.flush, ent); AL(W.reset, ent); AL(W.finish, ent);
  AL(W.L11, ent * kPanel * kPanel); AL(W.Dblk, ent * 2 * kPanel); AL(W.pi, ent * kPanel);
  AL(W.pt, ent * kPanel); AL(W.colmax, ent * kPanel);
  c->W0 = W;
  c->w_cap_entries = W.cap;
  AL(c->d_cbpool, P.cb_total);
  AL(c->d_red, 6 * kMaxShifts);
  AL(c->d_flops, KC_COUNT + 1);
  if (cudaMemset(c->d_flops, 0, sizeof(unsigned long long) * (KC_COUNT + 1)) != cudaSuccess) { kep_destroy(c); return KEP_ERR_CUDA; }
  AL(c->d_bnew, P.n); AL(c->d_xnew, P.n);
  AL(c->d_solve_partial, static_cast<size_t>(c->num_sms) * 4 * (kSolveBlk + 1));
  AL(c->d_df_ctr, 1 + 2 * static_cast<size_t>(P.nlevels));
  AL(c->d_io0, P.n); AL(c->d_io1, P.n); AL(c->d_io2, P.n); AL(c->d_io3, P.n); AL(c->d_io4, P.n);
#undef AL
  st = setup_memory(c);
  if (st != KEP_OK) { kep_destroy(c); return st; }
  if (cudaMallocHost(reinterpret_cast<void**>(&c->h_done), sizeof(int32_t) * ent) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&c->h_red), sizeof(long long) * 6 * kMaxShifts) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&c->h_df_err), sizeof(int32_t)) != cudaSuccess) {
    kep_destroy(c);
    return KEP_ERR_NOMEM;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { kep_destroy(c); return KEP_ERR_CUDA; }
  *out = c;
  return KEP_OK;
}

kep_status kep_get_info(const kep_ctx* c, kep_info* info) {
  if (!c || !info) return KEP_ERR_INVALID;
  const Plan& P = c->plan;
  info->n = P.n;
  info->nnz = P.nnz;
  info->nfronts = P.nfronts;
  info->nlevels = P.nlevels;
  info->max_front = P.max_front;
  info->nnz_factor = P.nnz_factor;
  info->flops_factor = P.flops;
  info->front_bytes = P.front_total * 8;
  info->replans = c->replans;
  info->cb_bytes = P.cb_total * 8;
  info->slot_bytes = shift_bytes(P);
  return KEP_OK;
}

kep_status kep_symbolic_info(int64_t n, const int64_t* rowptr, const int32_t* colind, int flags,
                             const double* coords, kep_info* info) {
  if (!info) return KEP_ERR_INVALID;
  FullPattern FP;
  const kep_status ps = full_pattern(n, rowptr, colind, nullptr, nullptr, (flags & KEP_PATTERN_LOWER) != 0, FP);
  if (ps != KEP_OK) return ps;
  Plan P;
  std::string err;
  const kep_status st = build_plan(n, FP.cnt, FP.ci, FP.av, FP.bv, coords, (flags & KEP_ORDER_GRAPH) != 0, (flags & KEP_ORDER_REFINED) != 0,
                                   false, 8, P, err);
  if (st != KEP_OK) return st;
  info->n = P.n;
  info->nnz = P.nnz;
  info->nfronts = P.nfronts;
  info->nlevels = P.nlevels;
  info->max_front = P.max_front;
  info->nnz_factor = P.nnz_factor;
  info->flops_factor = P.flops;
  info->front_bytes = P.front_total * 8;
  info->replans = 0;
  info->cb_bytes = P.cb_total * 8;
  info->slot_bytes = shift_bytes(P);
  return KEP_OK;
}

kep_status kep_set_stream(kep_ctx* c, void* stream) {
  if (!c) return KEP_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return KEP_OK;
}

kep_status kep_set_schur_mode(kep_ctx* c, int mode, int64_t min_front) {
  if (!c || (mode != KEP_SCHUR_FP64 && mode != KEP_SCHUR_EMULATED && mode != KEP_SCHUR_FP32) || min_front < 1)
    return KEP_ERR_INVALID;
  c->schur_mode = mode;
  c->emul_min_front = min_front;
  return KEP_OK;
}

kep_status kep_set_schur_tile(kep_ctx* c, int edge) {
  if (!c || (edge != 32 && edge != 64)) return KEP_ERR_INVALID;
  c->schur_tile = edge;
  return KEP_OK;
}

kep_status kep_get_schur_config(const kep_ctx* c, int* mode, int64_t* min_front, int* tile) {
  if (!c) return KEP_ERR_INVALID;
  if (mode) *mode = c->schur_mode;
  if (min_front) *min_front = c->emul_min_front;
  if (tile) *tile = c->schur_tile;
  return KEP_OK;
}

kep_status kep_factor(kep_ctx* c, double sigma, kep_inertia* out) {
  return kep_factor_pencil(c, 1.0, -sigma, out);
}

kep_status kep_factor_pencil(kep_ctx* c, double ca, double cb, kep_inertia* out) {
  if (!c) return KEP_ERR_INVALID;
  if (!std::isfinite(ca) || !std::isfinite(cb)) return KEP_ERR_INVALID;
  return ctx_factor(c, 0, ca, cb, out);
}

kep_status kep_solve(kep_ctx* c, const double* rhs, double* x, int64_t nrhs, int ptr_kind) {
  if (!c || !rhs || !x || nrhs < 0) return KEP_ERR_INVALID;
  if (c->herm_n) return herm_solve(c, rhs, x, nrhs, ptr_kind);
  const int64_t n = c->plan.n;
  for (int64_t r = 0; r < nrhs; ++r) {
    const double* b = rhs + r * n;
    double* xr = x + r * n;
    kep_status st;
    if (ptr_kind == KEP_DEVICE) {
      st = ctx_solve_dev(c, 0, b, xr);
    } else {
      if (cudaMemcpyAsync(c->d_io0, b, n * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return KEP_ERR_CUDA;
      st = ctx_solve_dev(c, 0, c->d_io0, c->d_io1);
      if (st == KEP_OK &&
          cudaMemcpyAsync(xr, c->d_io1, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return KEP_ERR_CUDA;
    }
    if (st != KEP_OK) return st;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->timer.collect();
  return KEP_OK;
}

}  // extern "C"

namespace {
__global__ void axpby_kernel(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
__global__ void __launch_bounds__(256) absmax_kernel(int64_t n, const double* x, double* partial) {
  __shared__ double red[8];
  double m = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    partial[blockIdx.x] = fmax(m, red[0]);
  }
}
}  // namespace

// y = a x + b y on the device (ctx's stream)
static kep_status vec_axpby_dev(kep_ctx* c, double a, const double* x, double b, double* y) {
  const int64_t n = c->plan.n;
  const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 4, (n + 255) / 256)));
  KEP_LAUNCH(&c->timer, KC_VEC, c->stream, axpby_kernel<<<g, 256, 0, c->stream>>>(n, a, x, b, y));
  return cudaGetLastError() == cudaSuccess ? KEP_OK : KEP_ERR_CUDA;
}

// max |x_i| (synchronises the stream)
static kep_status vec_norm_inf_dev(kep_ctx* c, const double* x, double* out) {
  const int64_t n = c->plan.n;
  const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 4, (n + 255) / 256)));
  KEP_LAUNCH(&c->timer, KC_VEC, c->stream, absmax_kernel<<<g, 256, 0, c->stream>>>(n, x, c->d_solve_partial));
  std::vector<double> h(g);
  if (cudaMemcpyAsync(h.data(), c->d_solve_partial, g * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return KEP_ERR_CUDA;
  double m = 0.0;
  for (double v : h) m = std::max(m, v);
  *out = m;
  return KEP_OK;
}

// y = (ca A + cb B) x for the pencil of the last factor (device vectors; t1: scratch)
static kep_status pencil_apply(kep_ctx* c, const double* x, double* y, double* t1) {
  KEP_TRY(ctx_spmv_dev(c, x, y, t1));
  const FactorSlot& S = c->slot[0];
  return vec_axpby_dev(c, S.cb, t1, S.ca, y);
}

// Iterative refinement with the factor in slot 0, device vectors (b is not modified; scratch:
// d_io2, d_io3 and the context's Krylov workspace, allocated at first use).
//
// GMRES-based refinement (Carson and Higham, SIAM J. Sci. Comput. 39(6), 2017), in the right-
// preconditioned flexible form (Saad, SIAM J. Sci. Comput. 14(2), 1993): every outer step takes
// the residual r = b - M x in FP64 and runs up to kGmresRestart Arnoldi steps on M S^{-1}, S the
// (reduced-precision) factor, with classical Gram-Schmidt applied twice and Givens rotations for
// the least-squares problem; then x += Z y, Z = S^{-1} V.  Plain refinement, x += S^{-1} r, only
// contracts while ||I - S^{-1} M|| < 1, which fails for the nearly singular shifted matrices of
// Algorithm 3 (an eigenvalue within the factor's perturbation of sigma); S^{-1} M then has a few
// outlying eigenvalues, and GMRES removes each in about one step.
namespace {
constexpr int kGmresRestart = 20;
}

kep_status kep::ctx_solve_refined_dev(kep_ctx* c, const double* b, double* xd, double tol, int32_t max_iter,
                                      int32_t* iters, double* berr) {
  const FactorSlot& S = c->slot[0];
  if (!c->slot_ready[0] || !S.valid) return KEP_ERR_INVALID;
  const int64_t n = c->plan.n;
  constexpr int m = kGmresRestart;
  const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->num_sms * 4, (n + 255) / 256)));
  if (!c->d_krylov) {          // V: (m + 1) n, Z: m n, dot partials, coefficients
    const size_t cnt = static_cast<size_t>(2 * m + 1) * n + static_cast<size_t>(nb) * (m + 1) + (m + 1);
    double* p = nullptr;
    if (cudaMalloc(&p, cnt * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return KEP_ERR_NOMEM; }
    c->allocs.push_back(p);
    c->d_krylov = p;
  }
  double* V = c->d_krylov;
  double* Z = V + static_cast<size_t>(m + 1) * n;
  double* part = Z + static_cast<size_t>(m) * n;
  double* coef = part + static_cast<size_t>(nb) * (m + 1);
  VecOps ops;
  ops.n = n; ops.num_blocks = nb; ops.partial = part; ops.stream = c->stream; ops.timer = &c->timer;
  auto host = [&](double* h, int cnt) -> kep_status {
    if (cudaMemcpyAsync(h, coef, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    return KEP_OK;
  };
  double *r = c->d_io2, *t = c->d_io3;
  // ||M||_inf bound for the backward error: |ca| ||A||_inf + |cb| ||B||_inf
  const double norm_m = std::fabs(S.ca) * c->plan.norm_a_inf + std::fabs(S.cb) * c->norm_b_inf;
  KEP_TRY(ctx_solve_dev(c, 0, b, xd));
  double bn;
  KEP_TRY(vec_norm_inf_dev(c, b, &bn));
  double eta = 0.0;
  int32_t it = 0;
  std::vector<double> H(static_cast<size_t>(m + 1) * m), g(m + 1), cs(m), sn(m), h(m + 1), h2(m + 1), y(m);
  while (true) {
    KEP_TRY(pencil_apply(c, xd, r, t));                  // r = M x
    KEP_TRY(vec_axpby_dev(c, 1.0, b, -1.0, r));          // r = b - M x
    double rn, xn;
    KEP_TRY(vec_norm_inf_dev(c, r, &rn));
    KEP_TRY(vec_norm_inf_dev(c, xd, &xn));
    eta = rn / (norm_m * xn + bn);
    if (!(eta > tol) || it >= max_iter) break;
    ops.dots(r, n, 1, r, coef);
    double beta2;
    KEP_TRY(host(&beta2, 1));
    const double beta = std::sqrt(beta2);
    if (!(beta > 0.0) || !std::isfinite(beta)) break;
    ops.axpby(1.0 / beta, r, 0.0, V);                   // v_0 = r / beta
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    // ||r||_inf <= ||r||_2: stop the inner steps once the 2-norm estimate meets the target
    const double target = tol * (norm_m * xn + bn);
    int k = 0;
    for (int j = 0; j < m && it < max_iter; ++j) {
      double* vj = V + static_cast<size_t>(j) * n;
      double* zj = Z + static_cast<size_t>(j) * n;
      double* w = V + static_cast<size_t>(j + 1) * n;
      KEP_TRY(ctx_solve_dev(c, 0, vj, zj));              // z_j = S^{-1} v_j
      KEP_TRY(pencil_apply(c, zj, w, t));                // w = M z_j
      for (int pass = 0; pass < 2; ++pass) {             // classical Gram-Schmidt, twice
        ops.dots(V, n, j + 1, w, coef);
        KEP_TRY(host(pass == 0 ? h.data() : h2.data(), j + 1));
        ops.combine(V, n, j + 1, coef, -1.0, 1.0, w);
      }
      for (int i = 0; i <= j; ++i) h[i] += h2[i];
      ops.dots(w, n, 1, w, coef);
      double hn2;
      KEP_TRY(host(&hn2, 1));
      const double hn = std::sqrt(hn2);
      h[j + 1] = hn;
      for (int i = 0; i < j; ++i) {                      // earlier rotations
        const double a0 = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = a0;
      }
      const double rr = std::hypot(h[j], h[j + 1]);
      cs[j] = rr == 0.0 ? 1.0 : h[j] / rr;
      sn[j] = rr == 0.0 ? 0.0 : h[j + 1] / rr;
      h[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[static_cast<size_t>(j) * (m + 1) + i] = h[i];
      ++it;
      k = j + 1;
      if (!(hn > 1e-300) || std::fabs(g[j + 1]) <= target) break;   // breakdown: the solution is exact
      ops.axpby(0.0, w, 1.0 / hn, w);
    }
    if (k == 0) break;
    for (int i = k - 1; i >= 0; --i) {                   // y = R^{-1} g (upper triangular)
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[static_cast<size_t>(q) * (m + 1) + i] * y[q];
      const double d = H[static_cast<size_t>(i) * (m + 1) + i];
      y[i] = d != 0.0 ? s / d : 0.0;
    }
    if (cudaMemcpyAsync(coef, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    ops.combine(Z, n, k, coef, 1.0, 1.0, xd);            // x += Z y
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;   // y is host memory
  }
  if (iters) *iters = it;
  if (berr) *berr = eta;
  return std::isfinite(eta) && eta <= tol ? KEP_OK : KEP_ERR_NOT_CONVERGED;
}

extern "C" {

kep_status kep_solve_refined(kep_ctx* c, const double* rhs, double* x, int ptr_kind, double tol, int32_t max_iter,
                             int32_t* iters, double* berr) {
  if (!c || !rhs || !x || tol < 0 || max_iter < 0) return KEP_ERR_INVALID;
  if (ptr_kind != KEP_HOST && ptr_kind != KEP_DEVICE) return KEP_ERR_INVALID;
  if (c->herm_n) return herm_solve_refined(c, rhs, x, ptr_kind, tol, max_iter, iters, berr);
  const int64_t n = c->plan.n;
  cudaStream_t st = c->stream;
  double *b = c->d_io0, *xd = c->d_io1;
  if (cudaMemcpyAsync(b, rhs, n * sizeof(double), ptr_kind == KEP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return KEP_ERR_CUDA;
  const kep_status rs = ctx_solve_refined_dev(c, b, xd, tol, max_iter, iters, berr);
  if (rs != KEP_OK && rs != KEP_ERR_NOT_CONVERGED) return rs;
  if (cudaMemcpyAsync(x, xd, n * sizeof(double), ptr_kind == KEP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return KEP_ERR_CUDA;
  c->timer.collect();
  return rs;
}

kep_status kep_spmv(kep_ctx* c, const double* x, double* ax, double* bx, int ptr_kind) {
  if (!c || !x || (!ax && !bx)) return KEP_ERR_INVALID;
  if (c->herm_n) return herm_spmv(c, x, ax, bx, ptr_kind);
  const int64_t n = c->plan.n;
  kep_status st;
  if (ptr_kind == KEP_DEVICE) {
    st = ctx_spmv_dev(c, x, ax, bx);
  } else {
    if (cudaMemcpyAsync(c->d_io0, x, n * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    st = ctx_spmv_dev(c, c->d_io0, ax ? c->d_io1 : nullptr, bx ? c->d_io2 : nullptr);
    if (st != KEP_OK) return st;
    if (ax && cudaMemcpyAsync(ax, c->d_io1, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
    if (bx && cudaMemcpyAsync(bx, c->d_io2, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return KEP_ERR_CUDA;
  }
  if (st != KEP_OK) return st;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->timer.collect();
  return KEP_OK;
}

kep_status kep_factor_multi(kep_ctx* c, const double* sigmas, int32_t ns, kep_inertia* out) {
  if (!c || !sigmas || !out || ns < 1) return KEP_ERR_INVALID;
  int G = ns > 1 ? multi_group(c, ns) : 1;
  if (G > 1) {
    const int ngroups = (ns + G - 1) / G;
    G = (ns + ngroups - 1) / ngroups;              // groups of (nearly) equal size
  }
  if (G <= 1) {
    for (int32_t i = 0; i < ns; ++i) {
      const kep_status st = kep_factor(c, sigmas[i], &out[i]);
      if (st != KEP_OK && st != KEP_ERR_SINGULAR) return st;
    }
    return KEP_OK;
  }
  for (int attempt = 0;; ++attempt) {
    bool redo = false;
    std::vector<const FactorSlot*> failed;
    for (int32_t q0 = 0; q0 < ns && !redo; q0 += G) {
      const int gs = static_cast<int>(std::min<int32_t>(G, ns - q0));
      KEP_TRY(alloc_slot(c, 0));
      const kep_status ms = ensure_multi(c, gs);
      if (ms == KEP_ERR_NOMEM && q0 == 0) {         // no room after all: one shift at a time
        cudaGetLastError();
        for (int32_t i = 0; i < ns; ++i) {
          const kep_status st = kep_factor(c, sigmas[i], &out[i]);
          if (st != KEP_OK && st != KEP_ERR_SINGULAR) return st;
        }
        return KEP_OK;
      }
      KEP_TRY(ms);
      FactorSlot* slots[kMaxShifts];
      double* pools[kMaxShifts];
      double* p21[kMaxShifts];
      double ca[kMaxShifts], cb[kMaxShifts];
      kep_inertia in[kMaxShifts];
      int bits[kMaxShifts];
      for (int j = 0; j < gs; ++j) {
        const bool last = j == gs - 1;             // the last shift ends in the public slot
        slots[j] = last ? &c->slot[0] : &c->mslot[j];
        pools[j] = last ? c->d_cbpool : c->mpool[j];
        p21[j] = last ? c->W.P21 : c->mp21[j];
        ca[j] = 1.0;
        cb[j] = -sigmas[q0 + j];
        bits[j] = 0;
      }
      KEP_TRY(factor_set(c, gs, slots, pools, p21, ca, cb, in, bits));
      for (int j = 0; j < gs; ++j) redo = redo || (bits[j] & ST_POOL);
      if (redo) {
        for (int j = 0; j < gs; ++j)
          if (bits[j] & ST_POOL) failed.push_back(slots[j]);
        break;
      }
      KEP_TRY(record_slot(c, 0, bits[gs - 1]));
      for (int j = 0; j < gs; ++j) {
        out[q0 + j] = in[j];
        kep_status st = finish_slot(c, *slots[j], in[j], bits[j]);
        if (j == gs - 1) c->slot_zero[0] = c->slot[0].valid ? in[j].zero : 0;
        st = herm_counts(c, st, &out[q0 + j]);
        if (st != KEP_OK && st != KEP_ERR_SINGULAR) return st;
      }
    }
    if (!redo) return KEP_OK;
    if (attempt >= 8) return KEP_ERR_POOL;
    KEP_TRY(replan(c, failed));
  }
}

kep_status kep_set_graphs(kep_ctx* c, int enable) {
  if (!c) return KEP_ERR_INVALID;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->graphs.enabled = enable != 0;
  return KEP_OK;
}

kep_status kep_set_timing(kep_ctx* c, int enable) {
  if (!c) return KEP_ERR_INVALID;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->timer.collect();
  c->timer.enabled = enable != 0;
  return KEP_OK;
}

kep_status kep_set_timing_classes(kep_ctx* c, unsigned int mask) {
  if (!c) return KEP_ERR_INVALID;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->timer.collect();
  c->timer.mask = mask;
  return KEP_OK;
}

kep_status kep_get_timing(kep_ctx* c, kep_timing* out, int reset) {
  if (!c || !out) return KEP_ERR_INVALID;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return KEP_ERR_CUDA;
  c->timer.collect();
  int64_t total = 0;
  unsigned long long fl[KC_COUNT + 1];
  if (cudaMemcpy(fl, c->d_flops, sizeof(fl), cudaMemcpyDeviceToHost) != cudaSuccess) return KEP_ERR_CUDA;
  for (int k = 0; k < KEP_NKCLASS; ++k) {
    out->launches[k] = c->timer.launches[k];
    out->ms[k] = c->timer.ms[k];
    out->flops[k] = static_cast<double>(fl[k]);
    total += c->timer.launches[k];
  }
  out->flush_fp64_equivalent_flops = static_cast<double>(fl[KC_COUNT]);
  out->total_launches = total;
  if (reset) {
    c->timer.reset();
    if (cudaMemset(c->d_flops, 0, sizeof(fl)) != cudaSuccess) return KEP_ERR_CUDA;
  }
  return KEP_OK;
}

void kep_destroy(kep_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  c->graphs.clear();
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->mem_allocs) cudaFree(p);
  if (c->h_done) cudaFreeHost(c->h_done);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->h_df_err) cudaFreeHost(c->h_df_err);
  c->driver_release();
  c->timer.release();
  delete c;
}

}  // extern "C"
