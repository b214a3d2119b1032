// Internal declarations of the kep library (host analysis plan, device layout, kernel launchers).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/kep.h"

namespace kep {

// ---------------------------------------------------------------------------------------------
// Tunables
// ---------------------------------------------------------------------------------------------
constexpr int kSmallMax = 128;      // fronts with m_alloc <= this are factored in shared memory
constexpr int kPanel = 32;          // block width of the large-front pivoting panel
constexpr int kWindow = 256;        // pivot window: the trailing matrix right of it is updated once
                                    //   per window with all of the window's pivots
constexpr int kSolveBigM = 512;     // fronts at least this large (and with kSolveBigP pivots) are
constexpr int kSolveBigP = 32;      //   solved by the dataflow path
constexpr int kSolveBlk = 64;       // row block of the dataflow solve
constexpr double kBKAlpha = 0.6403882032022076;   // (1 + sqrt 17) / 8
constexpr double kThresholdU = 0.01;               // threshold pivoting parameter u

// ---------------------------------------------------------------------------------------------
// Kernel launch accounting: every launch is counted per class; when enabled, each launch is
// bracketed by CUDA events on its stream and the elapsed times are summed at the next sync.
// ---------------------------------------------------------------------------------------------
enum KClass : int {
  KC_ASSEMBLE = 0, KC_PANEL, KC_L21, KC_APPLY, KC_UPDATE, KC_REDUCE,
  KC_SOLVE_FWD, KC_SOLVE_BWD, KC_PERM, KC_SPMV, KC_VEC, KC_SLICE, KC_FLUSH_TC, KC_COUNT
};

struct Timer {
  bool enabled = false;
  uint32_t mask = 0xffffffffu;        // classes timed while enabled
  int64_t launches[KC_COUNT] = {};
  double ms[KC_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> pending_cls;       // class of each recorded pair (events 2i, 2i+1)
  cudaEvent_t next_event() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  // record the start event of a launch of class cls (returns false when disabled)
  bool begin(int cls, cudaStream_t s) {
    ++launches[cls];
    if (!enabled || !((mask >> cls) & 1u)) return false;
    cudaEventRecord(next_event(), s);
    pending_cls.push_back(cls);
    return true;
  }
  void end(bool started, cudaStream_t s) {
    if (started) cudaEventRecord(next_event(), s);
  }
  // after the stream has synchronised: add up the recorded pairs and recycle the events
  void collect() {
    for (size_t i = 0; i < pending_cls.size(); ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) ms[pending_cls[i]] += t;
    }
    pending_cls.clear();
    used = 0;
  }
  void reset() {
    for (int c = 0; c < KC_COUNT; ++c) { launches[c] = 0; ms[c] = 0.0; }
  }
  void release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear(); used = 0; pending_cls.clear();
  }
};

#define KEP_LAUNCH(timer, cls, stream, ...)                  \
  do {                                                        \
    bool _kep_started = (timer)->begin((cls), (stream));      \
    __VA_ARGS__;                                              \
    (timer)->end(_kep_started, (stream));                     \
  } while (0)

// ---------------------------------------------------------------------------------------------
// Host-side symbolic plan (built once by kep_analyze, Section 3.3)
// ---------------------------------------------------------------------------------------------
struct Plan {
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> perm;    // perm[new] = old
  std::vector<int32_t> iperm;   // iperm[old] = new
  // assembly tree (fronts numbered in post-order: children before parents)
  int32_t nfronts = 0;
  std::vector<int32_t> first;       // first fully-summed variable (new numbering)
  std::vector<int32_t> p_sym;       // fully-summed count
  std::vector<int32_t> m_sym;       // front order without delays
  std::vector<int32_t> parent;      // -1 for a root
  std::vector<int32_t> child_ptr, child_idx;
  std::vector<int64_t> struct_ptr;  // struct_var[struct_ptr[t] .. +m_sym): fs vars then sorted CB vars
  std::vector<int32_t> struct_var;
  std::vector<int64_t> relmap_ptr;  // relmap[relmap_ptr[t] .. +(m_sym - p_sym)): parent position of
  std::vector<int32_t> relmap;      //   each symbolic CB row of t in the parent's symbolic struct
  std::vector<int64_t> ent_ptr;     // original lower entries owned by front t
  std::vector<int32_t> ent_r, ent_c;// symbolic (row, col) positions inside the front
  std::vector<double> ent_a, ent_b; // A and B values of those entries
  std::vector<int64_t> ent_src;     // position of each entry in the full symmetric CSR
  std::vector<int32_t> height;      // leaves 0
  int32_t nlevels = 0;
  std::vector<int32_t> level_ptr, level_fronts;   // fronts of each level, small ones first
  std::vector<int32_t> level_nsmall;              // count of small fronts per level
  std::vector<int32_t> level_nbig_solve;          // leading fronts of each level solved per block
  // memory plan.  Each front has persistent L storage (m_alloc x p_alloc, column-major,
  // ld = m_alloc: the fully-summed columns, later L and D) and a transient contribution block
  // (c x c, c = m_sym - p_sym, column-major) in a pool that lives from the front's factorization
  // until its parent's assembly.
  std::vector<int32_t> slack, m_alloc, p_alloc;
  std::vector<int64_t> front_off;   // doubles, L storage
  std::vector<int64_t> cb_off;      // doubles, contribution block in the pool (-1: none)
  std::vector<int64_t> vec_off;     // prefix of m_alloc (row lists, solve vectors)
  std::vector<int64_t> piv_off;     // prefix of p_alloc (D storage)
  int64_t front_total = 0, cb_total = 0, vec_total = 0, piv_total = 0;
  int64_t max_large_rows = 0;       // max over levels of sum of m_alloc of large fronts
  int32_t max_level_width = 0;
  std::vector<int64_t> p21_off;     // per front: offset of its L21 panel in the level workspace
  int32_t max_children = 0;
  int32_t slack_base = 0;
  // statistics
  int64_t max_front = 0, nnz_factor = 0;
  double flops = 0;
  double norm_a_inf = 0;            // ||A||_inf
};

// Build the plan from a full symmetric CSR pattern (both triangles, sorted, no duplicates).
// coords: optional n*3. graph_order forces the coordinate-free ordering; refined selects the
// cut search with minimum-vertex-cover separators; pairs orders rows r and r + n/2 together (the
// real embedding of a complex Hermitian pencil).
kep_status build_plan(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                      const std::vector<double>& av, const std::vector<double>& bv,
                      const double* coords, bool graph_order, bool refined, bool pairs, int32_t slack_base,
                      Plan& plan, std::string& err);

// kep_analyze flag used by kep_analyze_hermitian only: order the embedding's rows in pairs
constexpr int kOrderPairs = 1 << 20;

// (Re)compute the slack-dependent memory plan.
void plan_memory(Plan& plan, int32_t slack_base);
// Offsets and sizes of the slack-dependent storage from the per-front slack plan.slack.
void layout_memory(Plan& plan);

// ---------------------------------------------------------------------------------------------
// Device layout
// ---------------------------------------------------------------------------------------------
// Static per-front tables (uploaded once).
struct FrontTables {
  int32_t nfronts;
  const int32_t* first;
  const int32_t* p_sym;
  const int32_t* m_sym;
  const int32_t* m_alloc;
  const int32_t* parent;
  const int32_t* child_ptr;
  const int32_t* child_idx;
  const int64_t* struct_ptr;
  const int32_t* struct_var;
  const int64_t* relmap_ptr;
  const int32_t* relmap;
  const int64_t* ent_ptr;
  const int32_t* ent_r;
  const int32_t* ent_c;
  const double* ent_a;
  const double* ent_b;
  const int64_t* front_off;
  const int64_t* cb_off;
  const int64_t* vec_off;
  const int64_t* piv_off;
};



// One numeric factorization (a "slot"): dynamic per-front state + factor storage.
// d_in of a front whose storage could not take the delayed columns it received: -(need + 1), need
// the delayed columns it had to hold (0 when it failed because a child had failed)
struct FactorSlot {
  double* F;            // fronts (column-major, ld = m_alloc), lower triangle meaningful
  int32_t* rowvar;      // per front, m_alloc: variable (new numbering) at each factor position
  int32_t* apos;        // per front, m_alloc: assembly position of each factor position
  double* Dd;           // per front, p_alloc: diagonal of D
  double* De;           // per front, p_alloc: off-diagonal of a 2x2 block (at its first index)
  int8_t* piv;          // 1: 1x1, 2: first of a 2x2, 0: second of a 2x2
  int32_t* d_in;        // delayed columns received from the children
  int32_t* nelim;       // pivots eliminated in the front
  int32_t* d_out;       // fully-summed columns passed to the parent
  int32_t* cnt;         // per front: neg, zero, pos (3 ints)
  int32_t* status;      // [0]: error bits, [1]: first failing front
  double ca, cb;        // matrix factored: ca*A + cb*B
  bool valid = false;
};

// status bits
enum : int32_t {
  ST_POOL = 1,          // delays exceeded a front's slack
  ST_NONFINITE = 2,     // NaN/Inf pivot
  ST_ROOT_FORCED = 4,   // a root block failed the threshold test and was accepted as is
  ST_TIMEOUT = 8,       // a bounded wait inside a tensor-core kernel gave up
};

// Large-front step workspace (per level batch).
struct LargeWork {
  int32_t* list;        // fronts in the batch
  int32_t* k;           // eliminated so far
  int32_t* w;           // current block width
  int32_t* q;           // accepted in current block
  int32_t* fails;       // consecutive failed blocks
  int32_t* swap;        // pending move of a failed pivot (1 or 2 columns) to the end
  int32_t* ws;          // current pivot window [ws, we)
  int32_t* we;
  int32_t* kend;        // pivots [ws, kend) wait for the flush update
  int32_t* flush;       // 1: the flush update of the window is due this step
  int32_t* reset;       // 1: open a new window at the next pivot block
  int32_t* finish;      // 1: the front delays its remaining columns after the flush
  int32_t* done;        // 1 when the front has finished
  double* L11;          // per batch entry: kPanel*kPanel
  double* Dblk;         // per batch entry: 2*kPanel (diag, offdiag)
  int32_t* pi;          // per batch entry: kPanel local permutation
  int8_t* pt;           // per batch entry: kPanel pivot types
  unsigned long long* colmax;  // per batch entry: kPanel
  double* P21;          // per batch entry: rows x kPanel (offset p21_off)
  int64_t* p21_off;
  int32_t cap;          // capacity (entries)
};

// The factorizations one launch sequence serves: shift g of a multisection step factors
// ca[g] * A + cb[g] * B into slot s[g] with its own contribution-block pool and L21 workspace
// (g = 0 only for a single factorization).
constexpr int kMaxShifts = 8;
struct SlotSet {
  FactorSlot s[kMaxShifts];
  double* cbpool[kMaxShifts];
  double* P21[kMaxShifts];
  int32_t n;
};

// Entries of one tree level's launches: entry b is front lf[b] of shift sh[b] (sh null: shift 0).
struct Batch {
  const int32_t* lf;
  const int8_t* sh;
  int32_t e0;           // first entry of this batch within the level
};

// CUDA graphs of the factorization's step passes (one per level batch and pass length), replayed
// by later factorizations with the same storage; launch counts per class are replayed with them.
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int64_t launches[KC_COUNT] = {};
};
struct GraphCache {
  std::vector<std::pair<std::vector<uint64_t>, GraphEntry>> entries;
  bool enabled = true;
  GraphEntry* find(const std::vector<uint64_t>& key) {
    for (auto& e : entries) if (e.first == key) return &e.second;
    return nullptr;
  }
  void clear() {
    for (auto& e : entries) if (e.second.exec) cudaGraphExecDestroy(e.second.exec);
    entries.clear();
  }
};

struct FactorLaunch {
  const Plan* plan;
  FrontTables T;
  SlotSet SS;
  LargeWork W;
  int32_t G = 1;            // shifts: every level lists its fronts G times (front-major)
  const int32_t* d_ent_front;   // per entry (level-major, G entries per front): the front
  const int8_t* d_ent_shift;    //   and the shift (null for G = 1)
  const int32_t* h_ent_front;   // host copy
  int32_t* h_done;          // pinned, >= max level width x G
  long long* d_red;         // 6 entries per shift
  long long* h_red;         // pinned, 6 per shift
  cudaStream_t stream;
  int num_sms;
  Timer* timer;
  int64_t emul_min;         // fronts with m_alloc >= this use the tensor-core flush (0: never)
  bool fp32_schur = false;  // Schur tiles in FP32 arithmetic (reduced-precision factor for refined solves)
  int schur_tile = 64;      // edge of the FP64/FP32 Schur tiles: 32 or 64
  void* emul_ws;            // its workspace
  const int64_t* d_emul_off;      // per entry: byte offset of the entry's workspace in its batch
  const int32_t* h_emul_end;      // per entry starting a batch of such entries: its end (level-relative)
  unsigned long long* flops;   // per kernel class: algorithmic flops, counted on the device
  GraphCache* graphs = nullptr;   // step passes as CUDA graphs (null: direct launches)
  cudaStream_t capture_stream = nullptr;   // the stream the graphs are captured on
};

struct SolveLaunch {
  const Plan* plan;
  FrontTables T;
  FactorSlot S;
  const int32_t* d_level_fronts;
  const int32_t* d_perm;
  double* vasm;
  double* vfac;
  double* bnew;
  double* xnew;
  double* partial;            // num_sms * 4 * (kSolveBlk + 1) doubles (shared by a level's fronts)
  const int32_t* h_nelim;     // pivots eliminated per front (host copy of the factor's counts)
  // dataflow path (the leading level_nbig_solve[l] fronts of each level): work items of the
  // factorization (device) at per-level offsets (host, nlevels + 1 each)
  const int2* df_fwd_items;
  const int2* df_bwd_items;
  const int32_t* h_df_fwd_off;
  const int32_t* h_df_bwd_off;
  int32_t* df_counters;       // [0] wait error, [1, 1 + nlevels) forward, then backward counters
  int32_t* df_flags;          // per possible pivot block of every front (at df_fbase[front])
  const int32_t* df_fbase;
  int32_t epoch;              // this solve's number (flags compare against 2 epoch + 1 / + 2)
  double* df_part;            // backward partial sums of the contribution rows
  const int64_t* df_part_base;   // per front: its first partial sum
  int32_t* df_pcnt;           // per pivot block (at df_fbase): finished partial-sum chunks
  int64_t df_nflags;
  cudaStream_t stream;
  int num_sms;
  Timer* timer;
};

// Factor the G factorizations of F.SS (shift g: ca[g] A + cb[g] B); out[g], status_bits[g] per shift.
kep_status run_factor(FactorLaunch& F, const double* ca, const double* cb, kep_inertia* out, int* status_bits);
size_t emul_workspace_bytes(int64_t cap_rows);
void emul_init();
// low: the reduced-precision splitting (4 digits, KEP_SCHUR_FP32) instead of the FP64-accurate one
void launch_emul_update(bool window, bool low, const FrontTables& T, const SlotSet& SS, const LargeWork& W,
                        const Batch& B, int32_t nb, void* ws, const int64_t* d_off, int64_t rows_hint,
                        cudaStream_t st, int num_sms, Timer* timer, unsigned long long* flops);
int32_t emul_max_batch();
kep_status run_solve(SolveLaunch& L, const double* b, double* x);
void build_df_items(const Plan& P, const int32_t* nelim, const int32_t* din, std::vector<int2>& items,
                    std::vector<int32_t>& fwd_off, std::vector<int32_t>& bwd_off, int64_t& bwd_start,
                    std::vector<int64_t>& part_base, int64_t& part_total);
int64_t df_flag_bases(const Plan& P, std::vector<int32_t>& fbase);
kep_status run_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* a, const double* b,
                    const double* x, double* ya, double* yb, cudaStream_t st, int num_sms,
                    Timer* timer);

}  // namespace kep
