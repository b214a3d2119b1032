// The kep_ctx object behind the opaque C handle (library-internal).
#pragma once

#include <cmath>
#include <vector>

#include "kep_internal.h"

// return a non-OK status to the caller
#define KEP_TRY(x) do { kep_status _s = (x); if (_s != KEP_OK) return _s; } while (0)

struct kep_ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  kep::Plan plan;
  std::vector<void*> allocs;        // cudaMallocs that live as long as the context
  std::vector<void*> mem_allocs;    // cudaMallocs that depend on the slack plan (redone on re-plan)
  int replans = 0;
  kep::FrontTables T{};
  int32_t* d_level_fronts = nullptr;
  int32_t* d_perm = nullptr;
  int32_t* d_iperm = nullptr;
  // full symmetric CSR (original numbering) for the sparse products
  int64_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  double* d_a = nullptr;
  double* d_b = nullptr;
  // the caller's layout (kep_analyze's CSR) against that pattern
  int64_t nnz_in = 0;
  bool lower_in = false;
  std::vector<int64_t> csr_src;     // per full-CSR position: the caller's entry it came from
  int64_t* d_in2csr = nullptr;      // per caller entry: its full-CSR position (bit 62: a lower
                                    //   off-diagonal entry standing for both triangles)
  // a complex Hermitian pencil of order herm_n held as its real symmetric embedding of order
  // 2 herm_n (kep_analyze_hermitian); 0 for a real pencil
  int64_t herm_n = 0;
  int64_t herm_nnz = 0;             // the caller's stored complex entries
  bool herm_lower = false;
  int32_t* d_hrow = nullptr;        // per caller entry: row, column (in allocs)
  int32_t* d_hcol = nullptr;
  std::vector<int64_t> herm_emb_src;  // per entry given to the real analysis: the caller's entry
  std::vector<int8_t> herm_emb_part;  //   and the part it holds: 0 Re, +1 Im, -1 -Im
  // factorization slots: 0 = the public "last factor" (kep_factor / kep_solve),
  // 1 = the factor of B kept by the eigenpair driver during stage 1
  kep::FactorSlot slot[2]{};
  bool slot_ready[2] = {false, false};
  int slot_status[2] = {0, 0};
  int64_t slot_zero[2] = {0, 0};
  double* d_cbpool = nullptr;
  kep::LargeWork W{};
  kep::LargeWork W0{};              // W's entry arrays as allocated by kep_analyze (one shift)
  kep::GraphCache graphs;           // step passes of the factorization as CUDA graphs
  cudaStream_t capture_stream = nullptr;   // private stream the graphs are captured on
  long long* d_red = nullptr;
  unsigned long long* d_flops = nullptr;   // per kernel class (+1: FP64 work the tensor flush stands for)
  long long* h_red = nullptr;       // pinned
  int32_t* h_done = nullptr;        // pinned
  // solve workspaces
  double* d_vasm = nullptr;
  double* d_vfac = nullptr;
  double* d_bnew = nullptr;
  double* d_xnew = nullptr;
  double* d_io0 = nullptr;
  double* d_io1 = nullptr;
  double* d_io2 = nullptr;
  double* d_io3 = nullptr;
  double* d_io4 = nullptr;
  double norm_b_inf = 0;            // ||B||_inf
  double* d_krylov = nullptr;       // refinement workspace (in allocs; allocated at first use)
  double* d_solve_partial = nullptr;
  std::vector<int32_t> slot_nelim[2];   // pivots eliminated per front, per slot (host copy)
  std::vector<int32_t> slot_din[2];     // delayed columns received per front, per slot (host copy)
  uint64_t factor_version[2] = {0, 0};  // bumped by every successful factorization of the slot
  // dataflow solve: work items per slot (built from the slot's factorization), counters, flags
  uint64_t df_version[2] = {0, 0};
  std::vector<int2> df_items[2];
  std::vector<int32_t> df_fwd_off[2], df_bwd_off[2];
  int64_t df_bwd_start[2] = {0, 0};
  int2* d_df_items[2] = {nullptr, nullptr};   // in mem_allocs
  int64_t df_items_cap[2] = {0, 0};
  int32_t* d_df_ctr = nullptr;          // 1 + 2 nlevels (in allocs)
  int32_t* d_df_flags = nullptr;        // in mem_allocs
  int32_t* d_df_pcnt = nullptr;         // in mem_allocs, as many as the flags
  int64_t df_nflags = 0;
  std::vector<int64_t> df_part_base[2];
  int64_t* d_df_part_base[2] = {nullptr, nullptr};   // in mem_allocs (nfronts each)
  double* d_df_part = nullptr;          // in mem_allocs
  int64_t df_part_cap = 0;
  int32_t* d_df_fbase = nullptr;        // in mem_allocs
  int32_t* h_df_err = nullptr;          // pinned
  int32_t df_epoch = 0;
  kep::Timer timer;
  int schur_mode = KEP_SCHUR_EMULATED;
  int64_t emul_min_front = 512;
  int schur_tile = 64;              // edge of the FP64/FP32 Schur tiles (kep_set_schur_tile)
  void* emul_ws = nullptr;          // tensor-core update workspace (in mem_allocs)
  int64_t emul_bytes = 0;           // its size
  // multisection: G shifts factored in the same launches (kep_factor_multi).  Shift G - 1 uses
  // slot 0; shifts 0 .. G - 2 use their own slots, contribution-block pools and L21 workspaces
  // (in mem_allocs).  Entry lists: per level, each front G times (front-major).
  int32_t multi_cap = 0;            // shifts the extra resources serve (0: none)
  kep::FactorSlot mslot[kep::kMaxShifts]{};
  double* mpool[kep::kMaxShifts] = {};
  double* mp21[kep::kMaxShifts] = {};
  int32_t ent_G = 0;                // G the entry lists below were built for
  int32_t* d_ent_front = nullptr;   // (in mem_allocs)
  int8_t* d_ent_shift = nullptr;
  std::vector<int32_t> h_ent_front;
  int32_t w_cap_entries = 0;        // entries the LargeWork arrays hold
  // tensor-core batches, per G (1 and the multisection G): workspace offsets per entry, batch ends
  struct EmulPlan {
    int64_t min_planned = -1;
    int32_t G = 0;
    std::vector<int32_t> h_end;
    int64_t* d_off = nullptr;       // (in mem_allocs)
  } emul_plan[2];
  // eigenpair driver state (owned by driver.cu)
  void* driver = nullptr;
  void driver_release();
};

namespace kep {
kep_status ctx_factor(kep_ctx* c, int slot, double ca, double cb, kep_inertia* out);
kep_status ctx_solve_dev(kep_ctx* c, int slot, const double* b, double* x);
kep_status ctx_spmv_dev(kep_ctx* c, const double* x, double* ax, double* bx);
kep_status ctx_solve_refined_dev(kep_ctx* c, const double* b, double* x, double tol, int32_t max_iter,
                                 int32_t* iters, double* berr);
// Hermitian contexts: the public vector calls with complex vectors (interleaved re, im)
kep_status herm_solve(kep_ctx* c, const double* rhs, double* x, int64_t nrhs, int ptr_kind);
kep_status herm_spmv(kep_ctx* c, const double* x, double* ax, double* bx, int ptr_kind);
kep_status herm_solve_refined(kep_ctx* c, const double* rhs, double* x, int ptr_kind, double tol, int32_t max_iter,
                              int32_t* iters, double* berr);
kep_status herm_grad(kep_ctx* c, double lambda, const double* x, double lambda_bar, double* ga, double* gb,
                     int ptr_kind);
kep_status set_values_real(kep_ctx* c, const double* a_val, const double* b_val);
kep_status herm_set_values(kep_ctx* c, const double* a_val, const double* b_val);
// interleaved (re, im) complex vector of order herm_n <-> the embedding's [re; im] (device)
kep_status herm_to_blocked(kep_ctx* c, const double* in, double* out);
kep_status herm_to_interleaved(kep_ctx* c, const double* in, double* out);
}  // namespace kep
