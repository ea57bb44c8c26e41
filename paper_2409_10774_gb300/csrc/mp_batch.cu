// Batched and served solves (mp_batch_solve, mp_server_*).
//
// Many cells (RVEs), each with its own grid, phases and load path, advance
// together: every round runs ONE fixed-point iteration (Algorithm 2's loop
// body) of every cell that is iterating, as multi-cell launches of the same
// kernels mp_solve uses (y transform, z transform + Green operator, pass A
// with Algorithm 1, error reduction), preceded by the commits of cells whose
// increment converged in the previous round and the starts of their next
// increments.  Rounds run in windows of kRoundWindow, launched back to back
// with each cell's loop test taken on the device (RoundCtl) and replayed on
// the host from the window's error rows; a cell whose loop ended skips the
// rest of its window.  Each cell decides its own loop exit from its own error, so a
// cell's iterate sequence is exactly the one it has when solved alone: its
// work items are processed by whichever block picks them up, but every
// per-cell reduction (iteration error, homogenized averages) is folded from
// per-item records in item order, so its results do not depend on which other
// cells share the launches.
//
// Device memory: each resident cell owns one arena (state, tables, partial
// records, per-increment result rows, and the FP64 field buffer when the
// request wants fields), taken from a Pool.  The batch call takes arenas from
// the context's allocator; the server carves them from one block reserved at
// creation, whose size is its HBM budget: a request is admitted when its
// arena fits (requests wait in arrival order).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "../../include/micropolar.h"
#include "mp_host.cuh"
#include "mp_kernels.cuh"

using namespace mp;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ------------------------------------------------------------------ requests
// A validated, deep-copied problem and its outcome.
struct Request {
  uint64_t ticket = 0;
  int precision = 1;
  int n[3] = {1, 1, 1};
  double h = 1.0;
  long long nvox = 0;
  std::vector<uint16_t> phase;
  std::vector<mp_phase> phases;
  int n_steps = 0;
  std::vector<double> time, E, G;
  double tol = 1e-6, div_limit = 1e6;
  int err_kind = 0, max_iter = 10000;
  std::vector<int> lockstep;
  std::vector<double> tau_m, mu_m;  // manufactured source ((n_steps + 1) * nvox * 9 each), or empty
  double ref[6] = {0, 0, 0, 0, 0, 0};
  mp_result* res = nullptr;  // caller's host buffers (written when the solve ends)
  bool want_fields = false;
  size_t footprint = 0;      // arena bytes
  mp_status status = MP_OK;
  std::string message;
  bool done = false;
  std::chrono::steady_clock::time_point t_submit;
};

mp_status make_request(const mp_problem* p, mp_result* res, Request& q) {
  std::vector<long long> counts;
  mp_status st = validate_problem(p, &counts, q.ref, q.message);
  if (st != MP_OK) return st;
  q.precision = p->precision;
  for (int j = 0; j < 3; ++j) q.n[j] = p->n[j];
  q.h = p->h;
  q.nvox = (long long)p->n[0] * p->n[1] * p->n[2];
  q.phase.assign(p->phase, p->phase + q.nvox);
  q.phases.assign(p->phases, p->phases + p->n_phases);
  q.n_steps = p->n_steps;
  q.time.assign(p->time, p->time + p->n_steps + 1);
  q.E.assign(p->E, p->E + 9 * (size_t)(p->n_steps + 1));
  q.G.assign(p->G, p->G + 9 * (size_t)(p->n_steps + 1));
  q.tol = p->tol;
  q.err_kind = p->err_kind;
  q.max_iter = p->max_iter > 0 ? p->max_iter : 10000;
  if (p->lockstep_iters) q.lockstep.assign(p->lockstep_iters, p->lockstep_iters + p->n_steps);
  if (p->tau_m) {
    const size_t nsrc = (size_t)(p->n_steps + 1) * (size_t)q.nvox * 9;
    q.tau_m.assign(p->tau_m, p->tau_m + nsrc);
    q.mu_m.assign(p->mu_m, p->mu_m + nsrc);
  }
  q.div_limit = p->div_limit > 0 ? p->div_limit : 1e6;
  q.res = res;
  q.want_fields = res && (res->e || res->g || res->t || res->m || res->p || res->q);
  return MP_OK;
}

// ------------------------------------------------------------------ arena pools
struct Pool {
  virtual ~Pool() = default;
  virtual void* take(size_t bytes) = 0;  // nullptr when it does not fit
  virtual void give(void* p, size_t bytes) = 0;
};

// Arenas from the context's allocator.
struct CtxPool final : Pool {
  mp_ctx* ctx;
  explicit CtxPool(mp_ctx* c) : ctx(c) {}
  void* take(size_t bytes) override {
    DevBuf b;
    return dalloc(ctx, b, bytes) == MP_OK ? b.ptr : nullptr;
  }
  void give(void* p, size_t bytes) override {
    DevBuf b;
    b.ptr = p;
    b.bytes = bytes;
    dfree(ctx, b);
  }
};

// First-fit sub-allocation of one reserved block (free ranges kept sorted by
// offset and merged on release).
struct BlockPool final : Pool {
  unsigned char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_ranges;  // offset -> length
  BlockPool(void* b, size_t n) : base(static_cast<unsigned char*>(b)), size(n) {
    if (n) free_ranges[0] = n;
  }
  void* take(size_t bytes) override {
    bytes = align_up(bytes);
    for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_ranges.erase(it);
      if (len > bytes) free_ranges[off + bytes] = len - bytes;
      return base + off;
    }
    return nullptr;
  }
  void give(void* p, size_t bytes) override {
    bytes = align_up(bytes);
    size_t off = static_cast<unsigned char*>(p) - base;
    auto next = free_ranges.lower_bound(off);
    if (next != free_ranges.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_ranges.erase(next);
    }
    if (next != free_ranges.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_ranges[off] = bytes;
  }
};

// ------------------------------------------------------------------ cell arena layout
template <class R>
struct ArenaLayout {
  size_t spec, prev, hist, pq, elast, phase, phases, tw[3], status, tmean, ipart, apart, rows, src, fields, total;
  ArenaLayout(const Request& q, long long items_a) {
    const long long kx = q.n[0] > 1 ? q.n[0] / 2 : 1;
    const size_t nspec = (size_t)kx * q.n[1] * q.n[2];
    const size_t nv = (size_t)q.nvox;
    const size_t chunks = (nv + 255) / 256;
    size_t o = 0;
    auto put = [&](size_t bytes) {
      const size_t at = o;
      o += align_up(bytes);
      return at;
    };
    spec = put(sizeof(cpx<R>) * 18 * nspec);
    prev = put(sizeof(R) * 20 * nv);
    hist = put(sizeof(R) * 20 * nv);
    pq = put(sizeof(double) * 2 * nv);
    elast = put(sizeof(R) * 18 * nv);
    phase = put(sizeof(uint16_t) * nv);
    phases = put(sizeof(PhaseDev<R>) * q.phases.size());
    for (int a = 0; a < 3; ++a) tw[a] = put(sizeof(cpx<R>) * q.n[a]);
    status = put(sizeof(int) * 4);
    tmean = put(sizeof(double) * kCellScalars);
    ipart = put(sizeof(double) * kErrPartials * (size_t)items_a);
    apart = put(sizeof(double) * kAvgPartials * chunks);
    rows = put(sizeof(double) * kAvgPartials * (size_t)q.n_steps);
    src = put(q.tau_m.empty() ? 0 : sizeof(R) * 18 * nv * (size_t)q.n_steps);
    fields = q.want_fields ? put(sizeof(double) * 38 * nv) : o;
    total = o;
  }
};

// ------------------------------------------------------------------ engine
// Host-side progress of one cell through its load path (precision-free, so
// it moves with the cell between the FP32 and FP64 engines).
struct Progress {
  enum State { kInit, kStart, kIter, kCommit, kFinished };
  Request* req = nullptr;
  State state = kInit;
  int s = 1;  // current increment (1-based)
  int it = 0;
  double err = 0.0;
  mp_status step_status = MP_OK;
  bool predicted = false;
  int steps_done = 0, failed_step = 0;
  std::vector<double> err_steps;
  std::vector<int> iters_steps, iters64_steps;
  int it64 = 0;             // iterations of the current increment run in FP64
  double ref_err = 0.0;     // stagnation watch (FP32, stall_step): error level and
  int it_ref = 0;           //   iteration of its last new low, and the longest
  int gap = 0;              //   gap between lows in the increment
  int delta = 0;            // increment form: 0 off, 1 switching on this round, 2 on
  bool escalate = false;    // FP32 iteration stagnated: finish the increment in FP64
  bool demote = false;      // FP64-finished increment committed: next one in FP32
  bool restart = false;     // escalated: recompute the polarization of the current
                            // iterate and continue in the full form (in FP64)
  bool skip_delta = false;  // the increment form stalled once in this solve: later
                            // full-form stalls go to FP64 directly
};

// An FP32-mixed cell whose error has set no new low (a drop below kStallDrop times
// the last low) in kStallIters iterations while still above the tolerance has met the
// rounding floor of its FP32 transforms, which for strongly heterogeneous
// plastic cells can sit above the tolerance of the local error measure (a
// slowly but steadily converging cell keeps setting new lows and stays as it
// is).  It continues in the increment form, whose transforms round relative to
// the shrinking change of the polarization.
// That form removes the floor of the transforms, but not the one of the FP32
// stresses that enter the local error measure (a voxel's stress rounds at
// ~6e-8 of its own magnitude, which at stress concentrations can reach the
// tolerance relative to the mean): a cell that sets no new low for
// kStallItersDelta iterations there (or twice the longest gap between its
// earlier lows, so that a slow but steady contraction keeps going in FP32)
// finishes the increment in FP64.
// (The thresholds, kStallIters, kStallItersDelta and kStallDrop, are the
// single-cell solver's.)

// Iteration rounds per window: a window's launches run back to back on the
// device, each cell's loop test is taken there (RoundCtl) and the host
// reads the window's error rows once.  A cell whose loop ends inside a window
// idles for the window's remaining rounds (its commit waits for the window's
// end), so the window stays short against the typical increment.
constexpr int kRoundWindow = 8;

template <class R>
struct Slot {
  Progress g;
  unsigned char* arena = nullptr;
  size_t bytes = 0;
  CellDev<R> c{};
  LaunchCfg L;
  double* rows = nullptr;    // [n_steps][kAvgPartials] per-increment results
  double* fields = nullptr;  // [38][nvox] FP64 final fields (when requested)
  const R* src = nullptr;    // [n_steps][nvox][18] manufactured source, or NULL
};

template <class R>
class Engine;
template <class RA, class RB>
int migrate(Engine<RA>& from, Engine<RB>& to);

// Round-based multi-cell driver for one precision.
template <class R>
class Engine {
  template <class RA, class RB>
  friend int migrate(Engine<RA>& from, Engine<RB>& to);

 public:
  Engine(mp_ctx* ctx, Pool* pool, cudaStream_t st) : ctx_(ctx), pool_(pool), st_(st) {}
  ~Engine() {
    for (Slot<R>& s : slots_) release(s);
    slots_.clear();
    free_meta();
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (capture_) cudaStreamDestroy(capture_);
  }

  bool idle() const { return slots_.empty(); }
  size_t resident() const { return resident_; }
  int active() const { return (int)slots_.size(); }
  int64_t voxel_iters() const { return voxel_iters_; }
  int64_t rounds() const { return rounds_; }
  int64_t delta_switches() const { return delta_switches_; }

  // Arena bytes the request needs.
  size_t footprint(const Request& q) const {
    CellDev<R> c = shape_of(q);
    LaunchCfg L = make_launch_cfg<R>(c, ctx_->nsm);
    return ArenaLayout<R>(q, L.items_a).total;
  }

  // Allocates the cell's arena and uploads its tables.  MP_E_OOM when the
  // pool cannot hold it now (nothing is changed then).
  mp_status admit(Request* q) {
    Slot<R> s;
    s.g.req = q;
    mp_status st = build_slot(s, true);
    if (st != MP_OK) return st;
    s.g.state = Progress::kInit;
    resident_ += s.bytes;
    slots_.push_back(std::move(s));
    return MP_OK;
  }

  // Drops every resident request as MP_E_CANCELLED (arenas released).
  void cancel_all(std::vector<Request*>& finished) {
    for (Slot<R>& s : slots_) {
      s.g.req->status = MP_E_CANCELLED;
      s.g.req->message = "cancelled: the server was destroyed";
      finished.push_back(s.g.req);
      release(s);
    }
    slots_.clear();
  }

  // One window: the host's state changes (commits, starts), then up to
  // kRoundWindow iteration rounds.  Requests whose solve ended are appended
  // to `finished` (their results written, their arenas released).  A CUDA
  // failure fails every resident request and returns MP_E_CUDA.
  mp_status round(std::vector<Request*>& finished) {
    if (slots_.empty()) return MP_OK;
    ++rounds_;
    const int n = (int)slots_.size();
    constexpr bool kFp64 = sizeof(R) == 8;
    std::vector<int> l_commit, l_init, l_start, l_iter;
    for (int i = 0; i < n; ++i) {
      Slot<R>& sl = slots_[i];
      Progress& g = sl.g;
      CellDev<R>& c = sl.c;
      const Request& q = *g.req;
      c.err_out = nullptr;
      if (g.state == Progress::kCommit) {
        const bool predict = g.step_status == MP_OK && g.s < q.n_steps;
        c.predict = predict ? 1 : 0;
        c.ratio = predict ? (q.time[g.s + 1] - q.time[g.s]) / (q.time[g.s] - q.time[g.s - 1]) : 0.0;
        c.avg_out = sl.rows + (size_t)kAvgPartials * (g.s - 1);
        l_commit.push_back(i);
        g.predicted = predict;
        g.steps_done = g.s;
        if (g.step_status != MP_OK) {
          g.failed_step = g.s;
          g.state = Progress::kFinished;
        } else if (g.s == q.n_steps) {
          g.state = Progress::kFinished;
        } else {
          g.s += 1;
          g.state = Progress::kStart;
          // an FP32-mixed cell that finished this increment in FP64 starts the
          // next one in FP32 again (it moves after this round's commit)
          if (kFp64 && q.precision != 0) {
            g.demote = true;
            continue;
          }
        }
      }
      if (g.state == Progress::kInit || g.state == Progress::kStart) {
        for (int k = 0; k < 9; ++k) {
          c.E[k] = (R)q.E[9 * g.s + k];
          c.G[k] = (R)q.G[9 * g.s + k];
        }
        c.src = sl.src ? sl.src + (size_t)(g.s - 1) * (size_t)q.nvox * 18 : nullptr;
        if (g.state == Progress::kInit) l_init.push_back(i);
        l_start.push_back(i);
        g.state = Progress::kIter;
        g.it = 0;
        g.it64 = 0;
        g.delta = 0;
        g.err = 2.0 * q.tol;
        g.ref_err = 0.0;
        g.it_ref = 0;
        g.gap = 0;
      }
      if (g.state == Progress::kIter && g.restart) {
        // an escalated increment continues in FP64 in the full form: the
        // start pass forms the polarization of the current iterate (the
        // increment form's carried rounding is then damped, not kept)
        l_start.push_back(i);
        g.restart = false;
      }
      if (g.state == Progress::kIter) {
        c.delta_in = g.delta == 2 ? 1 : 0;
        c.delta_out = g.delta >= 1 ? 1 : 0;
        l_iter.push_back(i);
      }
    }
    // the window's loop control, one record per iterating cell
    const int K = l_iter.empty() ? 1 : kRoundWindow;
    mp_status st = ensure_meta(n);
    if (st != MP_OK) return fail_all(finished, st);
    RoundCtl* hctl = reinterpret_cast<RoundCtl*>(static_cast<unsigned char*>(h_meta_) + meta_.ctl);
    RoundCtl* dctl = reinterpret_cast<RoundCtl*>(static_cast<unsigned char*>(d_meta_) + meta_.ctl);
    double* derr = reinterpret_cast<double*>(static_cast<unsigned char*>(d_meta_) + meta_.err);
    for (int i = 0; i < n; ++i) slots_[i].c.rctl = nullptr;
    for (int i : l_iter) {
      Slot<R>& sl = slots_[i];
      const Progress& g = sl.g;
      const Request& q = *g.req;
      const int target = q.lockstep.empty() ? -1 : q.lockstep[g.s - 1];
      RoundCtl& rc = hctl[i];
      rc = RoundCtl{};
      rc.tol = q.tol;
      rc.div_limit = q.div_limit;
      rc.ref_err = g.ref_err;
      rc.rows = derr + (size_t)8 * kRoundWindow * i;
      rc.it = g.it;
      rc.target = target;
      rc.max_iter = q.max_iter;
      rc.it_ref = g.it_ref;
      rc.stag_iters = (!kFp64 && target < 0) ? (g.delta ? kStallItersDelta : kStallIters) : 0;
      rc.adapt = g.delta != 0 ? 1 : 0;
      rc.gap = g.gap;
      // the first round of the increment form changes the next round's inputs
      rc.max_rounds = (g.delta == 1) ? 1 : K;
      sl.c.rctl = dctl + i;
    }
    st = upload_and_launch(l_commit, l_init, l_start, l_iter, K);
    if (st != MP_OK) return fail_all(finished, st);
    rounds_ += K - 1;
    // decisions: the window's rows through Algorithm 2's loop test, per cell,
    // in round order (the device stopped each cell at its first decision)
    for (int i : l_iter) {
      Slot<R>& sl = slots_[i];
      Progress& g = sl.g;
      const RoundCtl& rc = hctl[i];
      const int ran = rc.rounds;
      bool iterating = true;
      bool agree = ran >= 1 && ran <= rc.max_rounds;
      for (int r = 0; agree && r < ran; ++r) {
        const double* e = h_err_ + (size_t)8 * (kRoundWindow * (size_t)i + r);
        iterating = decide(sl, e);
        if (!iterating && r != ran - 1) agree = false;
      }
      if (iterating && ran < rc.max_rounds) agree = false;
      if (!agree) {
        // the device's and the host's loop tests took different decisions
        g.step_status = MP_E_CUDA;
        g.failed_step = g.s;
        g.steps_done = g.s - 1;
        g.req->message = "internal: device and host loop decisions differ";
        g.state = Progress::kFinished;
      }
    }
    // harvest
    for (int i = 0; i < (int)slots_.size();) {
      if (slots_[i].g.state != Progress::kFinished) {
        ++i;
        continue;
      }
      Slot<R>& s = slots_[i];
      harvest(s);
      finished.push_back(s.g.req);
      release(s);
      slots_[i] = std::move(slots_.back());
      slots_.pop_back();
    }
    return MP_OK;
  }

 private:
  // Algorithm 2's loop test for one cell after one iteration whose error row
  // is e (err, four terms, status), with the FP32 stagnation watch.  Returns
  // true while the cell keeps iterating with an unchanged schedule; false when
  // its loop ended (it moves on to the commit, or finishes) or its schedule
  // changes (increment form switched on, or escalation to FP64).
  bool decide(Slot<R>& sl, const double* e) {
    constexpr bool kFp64 = sizeof(R) == 8;
    Progress& g = sl.g;
    const Request& q = *g.req;
    g.err = e[0];
    g.it += 1;
    if (kFp64) g.it64 += 1;
    if (g.delta == 1) g.delta = 2;  // this round wrote the first increment
    voxel_iters_ += q.nvox;
    const int target = q.lockstep.empty() ? -1 : q.lockstep[g.s - 1];
    mp_status out = MP_OK;
    bool leave = false;
    if (e[5] != 0.0) {
      out = MP_E_TIMEOUT;
      leave = true;
    } else if (!std::isfinite(g.err) || g.err > q.div_limit) {
      out = MP_E_DIVERGED;
      leave = true;
    } else {
      const bool more = target >= 0 ? g.it < target : g.err > q.tol;
      if (!more) {
        leave = true;
      } else if (target < 0 && g.it >= q.max_iter) {
        out = MP_E_NOT_CONVERGED;
        leave = true;
      }
    }
    if (!leave) {
      // FP32 stagnation watch (not under a prescribed iteration schedule)
      if (!kFp64 && target < 0) {
        if (stall_step(g.err, g.it, g.delta ? kStallItersDelta : kStallIters, g.delta != 0, g.ref_err, g.it_ref,
                       g.gap)) {
          if (g.delta == 0 && !g.skip_delta) {
            g.delta = 1;
            g.ref_err = g.err;
            g.it_ref = g.it;
            ++delta_switches_;
          } else {
            if (g.delta != 0) g.skip_delta = true;
            g.escalate = true;
          }
          return false;
        }
      }
      return true;
    }
    g.step_status = out;
    if (out == MP_E_TIMEOUT) {
      g.failed_step = g.s;
      g.steps_done = g.s - 1;
      g.state = Progress::kFinished;
    } else {
      g.err_steps.push_back(g.err);
      g.iters_steps.push_back(g.it);
      g.iters64_steps.push_back(g.it64);
      g.state = Progress::kCommit;
    }
    return false;
  }

  // Arena and device tables of the slot's request at this precision (rows
  // zeroed when fresh).
  mp_status build_slot(Slot<R>& s, bool fresh) {
    Request* q = s.g.req;
    s.c = shape_of(*q);
    s.L = make_launch_cfg<R>(s.c, ctx_->nsm);
    const ArenaLayout<R> A(*q, s.L.items_a);
    s.bytes = A.total;
    s.arena = static_cast<unsigned char*>(pool_->take(A.total));
    if (!s.arena) return MP_E_OOM;
    unsigned char* b = s.arena;
    CellDev<R>& c = s.c;
    c.spec = reinterpret_cast<cpx<R>*>(b + A.spec);
    c.prev = reinterpret_cast<R*>(b + A.prev);
    c.hist = reinterpret_cast<R*>(b + A.hist);
    c.pq = reinterpret_cast<double*>(b + A.pq);
    c.elast = reinterpret_cast<R*>(b + A.elast);
    c.phase = reinterpret_cast<const uint16_t*>(b + A.phase);
    c.phases = reinterpret_cast<const PhaseDev<R>*>(b + A.phases);
    c.status = reinterpret_cast<int*>(b + A.status);
    c.tmean = reinterpret_cast<double*>(b + A.tmean);
    c.ipart = reinterpret_cast<double*>(b + A.ipart);
    c.apart = reinterpret_cast<double*>(b + A.apart);
    c.rows_a = s.L.rows;
    c.items_a = s.L.items_a;
    s.rows = reinterpret_cast<double*>(b + A.rows);
    s.fields = q->want_fields ? reinterpret_cast<double*>(b + A.fields) : nullptr;
    c.ref = ref_dev<R>(q->ref);
    c.err_kind = q->err_kind;
    for (int k = 0; k < 9; ++k) {  // load of the current increment (a cell may move mid-increment)
      c.E[k] = (R)q->E[9 * s.g.s + k];
      c.src = nullptr;
      c.G[k] = (R)q->G[9 * s.g.s + k];
    }
    std::vector<PhaseDev<R>> ph(q->phases.size());
    for (size_t k = 0; k < ph.size(); ++k) ph[k] = phase_dev<R>(q->phases[k], q->precision == 2);
    AxisPlan<R>* plans[3] = {&c.px, &c.py, &c.pz};
    std::vector<cpx<R>> tw[3];
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3; ++a) {
      axis_tables<R>(q->n[a], a == 0, *plans[a], tw[a]);
      plans[a]->tw = reinterpret_cast<const cpx<R>*>(b + A.tw[a]);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + A.tw[a], tw[a].data(), sizeof(cpx<R>) * q->n[a], cudaMemcpyHostToDevice, st_);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b + A.phase, q->phase.data(), sizeof(uint16_t) * q->nvox, cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b + A.phases, ph.data(), sizeof(PhaseDev<R>) * ph.size(), cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + A.status, 0, sizeof(int) * 4, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + A.tmean, 0, sizeof(double) * kCellScalars, st_);
    if (e == cudaSuccess && fresh) e = cudaMemsetAsync(s.rows, 0, sizeof(double) * kAvgPartials * q->n_steps, st_);
    std::vector<R> src_host;
    if (!q->tau_m.empty()) {
      centred_source<R>(q->tau_m.data(), q->mu_m.data(), q->n_steps, q->nvox, src_host);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + A.src, src_host.data(), sizeof(R) * src_host.size(), cudaMemcpyHostToDevice, st_);
      s.src = reinterpret_cast<const R*>(b + A.src);
      c.src = s.src + (size_t)(s.g.s - 1) * (size_t)q->nvox * 18;
    }
    // the host tables above are locals: the copies must have read them
    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) {
      pool_->give(s.arena, s.bytes);
      s.arena = nullptr;
      q->message = std::string("admission: ") + cudaGetErrorString(e);
      return MP_E_CUDA;
    }
    return MP_OK;
  }

  CellDev<R> shape_of(const Request& q) const {
    CellDev<R> c{};
    c.n1 = q.n[0];
    c.n2 = q.n[1];
    c.n3 = q.n[2];
    c.kx = (c.n1 > 1) ? c.n1 / 2 : 1;
    c.nvox = q.nvox;
    c.nspec = (long long)c.kx * c.n2 * c.n3;
    c.h = q.h;
    c.inv_nvox = 1.0 / (double)q.nvox;
    for (int j = 0; j < 3; ++j) c.two_pi_over_L[j] = (R)(2.0 * M_PI / ((double)q.n[j] * q.h));
    return c;
  }

  void release(Slot<R>& s) {
    if (s.arena) {
      pool_->give(s.arena, s.bytes);
      resident_ -= s.bytes;
      s.arena = nullptr;
    }
  }

  // Metadata block (device and pinned host mirror): the descriptor table,
  // the per-family entry lists and item prefixes, and the error rows.
  struct Meta {
    size_t cells, act[6], pre[6], err, ctl, total;
  };
  Meta layout(int cap) const {
    Meta m;
    size_t o = 0;
    auto put = [&](size_t bytes) {
      const size_t at = o;
      o += align_up(bytes);
      return at;
    };
    m.cells = put(sizeof(CellDev<R>) * cap);
    for (int f = 0; f < 6; ++f) m.act[f] = put(sizeof(int) * cap);
    for (int f = 0; f < 6; ++f) m.pre[f] = put(sizeof(long long) * (cap + 1));
    m.err = put(sizeof(double) * 8 * kRoundWindow * cap);
    m.ctl = put(sizeof(RoundCtl) * cap);
    m.total = o;
    return m;
  }
  void free_meta() {
    if (d_meta_) cudaFree(d_meta_);
    if (h_meta_) cudaFreeHost(h_meta_);
    d_meta_ = h_meta_ = nullptr;
    h_err_ = nullptr;
    cap_ = 0;
  }
  mp_status ensure_meta(int n) {
    if (n <= cap_) return MP_OK;
    int cap = cap_ ? cap_ : 64;
    while (cap < n) cap *= 2;
    free_meta();
    const Meta m = layout(cap);
    if (cudaMalloc(&d_meta_, m.total) != cudaSuccess) {
      d_meta_ = nullptr;
      return MP_E_OOM;
    }
    if (cudaMallocHost(&h_meta_, m.total) != cudaSuccess) {
      h_meta_ = nullptr;
      return MP_E_OOM;
    }
    std::memset(h_meta_, 0, m.total);
    cap_ = cap;
    meta_ = m;
    return MP_OK;
  }

  enum Family { kFY = 0, kFZ, kFA, kFS, kFV, kFV0 };

  // One window: the commits and starts of this round, then `rounds`
  // iteration rounds of the cells in l_iter (each cell's loop test on the
  // device, its RoundCtl uploaded with the descriptors), then the window's
  // error rows and loop controls back to the host.
  mp_status upload_and_launch(const std::vector<int>& l_commit, const std::vector<int>& l_init,
                              const std::vector<int>& l_start, const std::vector<int>& l_iter, int rounds) {
    const int n = (int)slots_.size();
    mp_status st = ensure_meta(n);
    if (st != MP_OK) return st;
    unsigned char* hb = static_cast<unsigned char*>(h_meta_);
    unsigned char* db = static_cast<unsigned char*>(d_meta_);
    h_err_ = reinterpret_cast<double*>(hb + meta_.err);
    CellDev<R>* hc = reinterpret_cast<CellDev<R>*>(hb + meta_.cells);
    for (int i = 0; i < n; ++i) hc[i] = slots_[i].c;
    MultiCfg<R> m;
    long long* items[6] = {&m.items_y, &m.items_z, &m.items_a, &m.items_s, &m.items_v, &m.items_v0};
    Work<R>* works[6] = {&m.wy, &m.wz, &m.wa, &m.ws, &m.wv, &m.wv0};
    auto fill = [&](Family f, const std::vector<int>& list, auto count) {
      int* act = reinterpret_cast<int*>(hb + meta_.act[f]);
      long long* pre = reinterpret_cast<long long*>(hb + meta_.pre[f]);
      int k = 0;
      pre[0] = 0;
      for (int i : list) {
        const long long c = count(slots_[i]);
        if (c <= 0) continue;
        act[k] = i;
        pre[k + 1] = pre[k] + c;
        ++k;
      }
      Work<R>& w = *works[f];
      w.cells = reinterpret_cast<const CellDev<R>*>(db + meta_.cells);
      w.act = reinterpret_cast<const int*>(db + meta_.act[f]);
      w.pre = reinterpret_cast<const long long*>(db + meta_.pre[f]);
      w.n_act = k;
      *items[f] = pre[k];
    };
    fill(kFY, l_iter, [](const Slot<R>& s) { return s.c.n2 > 1 ? tiles_y(s.c) : 0ll; });
    fill(kFZ, l_iter, [](const Slot<R>& s) { return tiles_z(s.c); });
    fill(kFA, l_iter, [](const Slot<R>& s) { return s.c.items_a; });
    fill(kFS, l_start, [](const Slot<R>& s) { return s.c.items_a; });
    fill(kFV, l_commit, [](const Slot<R>& s) { return (s.c.nvox + 255) / 256; });
    fill(kFV0, l_init, [](const Slot<R>& s) { return (s.c.nvox + 255) / 256; });
    for (int i : l_iter) {
      const CellDev<R>& c = slots_[i].c;
      m.smem_y = std::max(m.smem_y, c.n2 > 1 ? smem_line_pass<R>(c.n2) : (size_t)0);
      m.smem_z = std::max(m.smem_z, smem_line_pass<R>(c.n3));
      m.smem_a = std::max(m.smem_a, smem_pass_a<R>(c.n1, c.rows_a));
    }
    for (int i : l_start) m.smem_a = std::max(m.smem_a, smem_pass_a<R>(slots_[i].c.n1, slots_[i].c.rows_a));
    multi_grids<R>(m, ctx_->nsm);
    // descriptors and lists, then the loop controls (the error rows between
    // them are device-written only)
    cudaError_t e = cudaMemcpyAsync(d_meta_, h_meta_, meta_.err, cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess && !l_iter.empty())
      e = cudaMemcpyAsync(db + meta_.ctl, hb + meta_.ctl, sizeof(RoundCtl) * n, cudaMemcpyHostToDevice, st_);
    if (e == cudaSuccess && !l_commit.empty()) e = launch_multi_commit<R>(m, st_);
    if (e == cudaSuccess && !l_start.empty()) e = launch_multi_start<R>(m, st_);
    if (e == cudaSuccess && !l_iter.empty()) e = launch_rounds(m, rounds);
    if (e == cudaSuccess && !l_iter.empty())
      e = cudaMemcpyAsync(h_err_, db + meta_.err, sizeof(double) * 8 * kRoundWindow * n, cudaMemcpyDeviceToHost,
                          st_);
    if (e == cudaSuccess && !l_iter.empty())
      e = cudaMemcpyAsync(hb + meta_.ctl, db + meta_.ctl, sizeof(RoundCtl) * n, cudaMemcpyDeviceToHost, st_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) {
      last_cuda_ = cudaGetErrorString(e);
      return MP_E_CUDA;
    }
    return MP_OK;
  }

  void harvest(Slot<R>& s) {
    const Progress& g = s.g;
    Request& q = *g.req;
    mp_result* res = q.res;
    q.status = (g.failed_step && g.step_status != MP_OK) ? g.step_status : MP_OK;
    if (q.status != MP_OK) {
      char buf[256];
      if (q.status == MP_E_TIMEOUT)
        std::snprintf(buf, sizeof(buf), "load increment %d: a bounded device wait expired", g.failed_step);
      else
        std::snprintf(buf, sizeof(buf), "load increment %d %s after %d iterations (err %.3e)", g.failed_step,
                      q.status == MP_E_DIVERGED ? "diverged" : "did not converge", g.it, g.err);
      q.message = buf;
    }
    if (!res) return;
    const int ns = g.steps_done;
    std::vector<double> rows((size_t)kAvgPartials * (ns > 0 ? ns : 1));
    cudaError_t e = cudaSuccess;
    if (ns > 0)
      e = cudaMemcpyAsync(rows.data(), s.rows, sizeof(double) * kAvgPartials * ns, cudaMemcpyDeviceToHost, st_);
    if (e == cudaSuccess && s.fields && ns > 0) {
      const size_t nv = (size_t)q.nvox;
      double* b = s.fields;
      double *fe = b, *fg = b + 9 * nv, *ft = b + 18 * nv, *fm = b + 27 * nv, *fp = b + 36 * nv, *fq = b + 37 * nv;
      e = launch_fields<R>(s.L, s.c, g.predicted ? 1 : 0, fe, fg, ft, fm, fp, fq, st_);
      struct {
        double* dst;
        double* src;
        size_t n;
      } cp[6] = {{res->e, fe, 9 * nv}, {res->g, fg, 9 * nv}, {res->t, ft, 9 * nv},
                 {res->m, fm, 9 * nv}, {res->p, fp, nv},     {res->q, fq, nv}};
      for (auto& x : cp)
        if (x.dst && e == cudaSuccess)
          e = cudaMemcpyAsync(x.dst, x.src, sizeof(double) * x.n, cudaMemcpyDeviceToHost, st_);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) {
      q.status = MP_E_CUDA;
      q.message = std::string("result copy: ") + cudaGetErrorString(e);
      return;
    }
    for (int k = 0; k < ns; ++k) {
      const double* row = rows.data() + (size_t)kAvgPartials * k;
      for (int c = 0; c < 9; ++c) {
        if (res->T) res->T[9 * k + c] = row[c];
        if (res->M) res->M[9 * k + c] = row[9 + c];
        if (res->Eavg) res->Eavg[9 * k + c] = row[18 + c];
        if (res->Gavg) res->Gavg[9 * k + c] = row[27 + c];
      }
      if (res->P) res->P[k] = row[36];
      if (res->Q) res->Q[k] = row[37];
      if (res->Teq) res->Teq[k] = row[38];
      if (res->Meq) res->Meq[k] = row[39];
      if (res->err) res->err[k] = g.err_steps[k];
      if (res->iters) res->iters[k] = g.iters_steps[k];
      if (res->iters_fp64) res->iters_fp64[k] = g.iters64_steps[k];
    }
    res->steps_done = ns;
    res->failed_step = g.failed_step;
    for (int i = 0; i < 6; ++i) res->ref_moduli_used[i] = q.ref[i];
  }

  mp_status fail_all(std::vector<Request*>& finished, mp_status st) {
    cudaStreamSynchronize(st_);  // no kernel of this round may still use an arena
    for (Slot<R>& s : slots_) {
      s.g.req->status = st;
      s.g.req->message = "device failure during a batched round: " + last_cuda_;
      finished.push_back(s.g.req);
      release(s);
    }
    slots_.clear();
    return st;
  }

  // The window's iteration rounds as one CUDA graph: captured for a launch
  // configuration (work lists, item counts, grids, shared memory, rounds) and
  // replayed while the configuration stays the same (the resident cells keep
  // iterating); the work lists' contents live in the metadata block, which
  // every window uploads before the launch.
  struct RoundsKey {
    Work<R> wy, wz, wa;
    long long items_y, items_z, items_a;
    size_t smem_y, smem_z, smem_a;
    int grid_y, grid_z, grid_a, rounds;
  };
  static RoundsKey rounds_key(const MultiCfg<R>& m, int rounds) {
    RoundsKey k;
    std::memset(&k, 0, sizeof(k));  // padding compares equal
    k.wy = m.wy;
    k.wz = m.wz;
    k.wa = m.wa;
    k.items_y = m.items_y;
    k.items_z = m.items_z;
    k.items_a = m.items_a;
    k.smem_y = m.smem_y;
    k.smem_z = m.smem_z;
    k.smem_a = m.smem_a;
    k.grid_y = m.grid_y;
    k.grid_z = m.grid_z;
    k.grid_a = m.grid_a;
    k.rounds = rounds;
    return k;
  }
  cudaError_t launch_rounds(const MultiCfg<R>& m, int rounds) {
    if (rounds <= 1) return launch_multi_iteration<R>(m, st_);
    const RoundsKey k = rounds_key(m, rounds);
    if (!(gexec_ && std::memcmp(&k, &gkey_, sizeof(k)) == 0)) {
      if (gexec_) cudaGraphExecDestroy(gexec_);
      gexec_ = nullptr;
      if (!capture_ && cudaStreamCreateWithFlags(&capture_, cudaStreamNonBlocking) != cudaSuccess) capture_ = nullptr;
      cudaGraph_t g = nullptr;
      cudaError_t e = capture_ ? cudaStreamBeginCapture(capture_, cudaStreamCaptureModeRelaxed)
                               : cudaErrorNotSupported;
      if (e == cudaSuccess) {
        cudaError_t el = cudaSuccess;
        for (int r = 0; r < rounds && el == cudaSuccess; ++r) el = launch_multi_iteration<R>(m, capture_);
        e = cudaStreamEndCapture(capture_, &g);
        if (e == cudaSuccess) e = el;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec_, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        // no graph: the same launches one by one
        cudaGetLastError();
        if (gexec_) cudaGraphExecDestroy(gexec_);
        gexec_ = nullptr;
        cudaError_t el = cudaSuccess;
        for (int r = 0; r < rounds && el == cudaSuccess; ++r) el = launch_multi_iteration<R>(m, st_);
        return el;
      }
      gkey_ = k;
    }
    return cudaGraphLaunch(gexec_, st_);
  }

  mp_ctx* ctx_;
  Pool* pool_;
  cudaStream_t st_;
  cudaStream_t capture_ = nullptr;
  cudaGraphExec_t gexec_ = nullptr;
  RoundsKey gkey_{};
  std::vector<Slot<R>> slots_;
  size_t resident_ = 0;
  int64_t voxel_iters_ = 0, rounds_ = 0, delta_switches_ = 0;
  void* d_meta_ = nullptr;
  void* h_meta_ = nullptr;
  double* h_err_ = nullptr;
  Meta meta_{};
  int cap_ = 0;
  std::string last_cuda_;
};

// Moves the flagged cells of `from` (FP32 cells whose iteration stagnated, or
// FP64-finished FP32-mixed cells about to start their next increment) to the
// engine of the other precision: the arena is rebuilt there and the state
// (iterate, history, plastic strains, predictor, result rows and, mid-
// increment, the polarization spectrum) is converted on the device.  A cell
// whose new arena does not fit stays where it is.  Returns the number moved.
template <class RA, class RB>
int migrate(Engine<RA>& from, Engine<RB>& to) {
  int moved = 0;
  for (size_t i = 0; i < from.slots_.size();) {
    Slot<RA>& src = from.slots_[i];
    const bool flagged = (sizeof(RA) == 4) ? src.g.escalate : src.g.demote;
    if (!flagged) {
      ++i;
      continue;
    }
    Slot<RB> dst;
    dst.g = src.g;
    if (src.g.escalate && src.g.state == Progress::kIter) {
      dst.g.delta = 0;
      dst.g.restart = true;
    }
    dst.g.escalate = dst.g.demote = false;
    if (to.build_slot(dst, false) != MP_OK) {
      src.g.escalate = src.g.demote = false;
      src.g.it_ref = src.g.it;  // watch again before the next attempt
      ++i;
      continue;
    }
    const Request& q = *src.g.req;
    const long long nv = q.nvox;
    cudaStream_t st = to.st_;
    const int nsm = to.ctx_->nsm;
    cudaError_t e = launch_convert<RA, RB>(src.c.prev, dst.c.prev, 20 * nv, nsm, st);
    if (e == cudaSuccess) e = launch_convert<RA, RB>(src.c.hist, dst.c.hist, 20 * nv, nsm, st);
    if (e == cudaSuccess) e = launch_convert<RA, RB>(src.c.elast, dst.c.elast, 18 * nv, nsm, st);
    if (e == cudaSuccess && src.g.state == Progress::kIter && !dst.g.restart)
      e = launch_convert<RA, RB>(reinterpret_cast<const RA*>(src.c.spec), reinterpret_cast<RB*>(dst.c.spec),
                                 36 * src.c.nspec, nsm, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst.c.pq, src.c.pq, sizeof(double) * 2 * nv, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst.c.tmean, src.c.tmean, sizeof(double) * kCellScalars, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst.rows, src.rows, sizeof(double) * kAvgPartials * q.n_steps, cudaMemcpyDeviceToDevice,
                          st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      to.pool_->give(dst.arena, dst.bytes);
      src.g.escalate = src.g.demote = false;
      src.g.it_ref = src.g.it;
      ++i;
      continue;
    }
    to.resident_ += dst.bytes;
    to.slots_.push_back(std::move(dst));
    from.release(src);
    from.slots_[i] = std::move(from.slots_.back());
    from.slots_.pop_back();
    ++moved;
  }
  return moved;
}

}  // namespace


// ================================================================== server
struct mp_server {
  mp_ctx* ctx = nullptr;
  mp_ctx wctx;  // the worker's copy (device, SM count): errors of the worker never touch ctx
  cudaStream_t stream = nullptr;
  DevBuf block;
  BlockPool* pool = nullptr;
  Engine<float>* ef = nullptr;
  Engine<double>* ed = nullptr;
  int max_resident = 1024;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // statistics, updated by the worker under `mu`
  int64_t submitted = 0, completed = 0, peak_resident = 0, resident = 0, rounds = 0, voxel_iters = 0;
  size_t resident_bytes = 0;
};

namespace {

int resident_count(const mp_server* S) { return S->ef->active() + S->ed->active(); }

void server_loop(mp_server* S) {
  cudaSetDevice(S->wctx.device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    // admission in arrival order while the head request fits
    while (!S->queue.empty() && !S->stop && resident_count(S) < S->max_resident) {
      Request* q = S->queue.front();
      lk.unlock();
      const bool idle = S->ef->idle() && S->ed->idle();
      mp_status st = q->precision == 0 ? S->ed->admit(q) : S->ef->admit(q);
      lk.lock();
      if (st == MP_E_OOM && !idle) break;  // wait until resident requests finish
      S->queue.pop_front();
      if (st != MP_OK) {
        q->status = st;
        if (q->message.empty()) q->message = "admission failed: the request does not fit the server's HBM budget";
        q->done = true;
        S->cv_done.notify_all();
      }
      S->resident = resident_count(S);
      S->resident_bytes = S->ef->resident() + S->ed->resident();
      if (S->resident > S->peak_resident) S->peak_resident = S->resident;
    }
    if (S->stop) break;
    if (S->ef->idle() && S->ed->idle()) {
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      continue;
    }
    lk.unlock();
    std::vector<Request*> fin;
    S->ef->round(fin);
    S->ed->round(fin);
    migrate(*S->ef, *S->ed);
    migrate(*S->ed, *S->ef);
    lk.lock();
    for (Request* q : fin) q->done = true;
    S->completed += (int64_t)fin.size();
    S->resident = resident_count(S);
    S->resident_bytes = S->ef->resident() + S->ed->resident();
    S->rounds = S->ef->rounds() + S->ed->rounds();
    S->voxel_iters = S->ef->voxel_iters() + S->ed->voxel_iters();
    if (!fin.empty()) S->cv_done.notify_all();
  }
  for (Request* q : S->queue) {
    q->status = MP_E_CANCELLED;
    q->message = "cancelled: the server was destroyed";
    q->done = true;
  }
  S->queue.clear();
  std::vector<Request*> fin;
  S->ef->cancel_all(fin);
  S->ed->cancel_all(fin);
  for (Request* q : fin) q->done = true;
  S->cv_done.notify_all();
}

}  // namespace

// ================================================================== C ABI
extern "C" {

mp_status mp_batch_solve(mp_ctx* ctx, const mp_problem* const* problems, int32_t count, mp_result* results,
                         mp_status* per_item, void* stream, mp_batch_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (!ctx) return set_error(nullptr, MP_E_INVALID_ARG, "ctx is NULL");
  if (count < 0 || (count > 0 && !problems)) return set_error(ctx, MP_E_INVALID_ARG, "invalid problem list");
  if (count == 0) return MP_OK;
  MP_DEVICE_SCOPE(ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  std::vector<Request> reqs((size_t)count);
  std::deque<Request*> pending;
  for (int i = 0; i < count; ++i) {
    Request& q = reqs[i];
    q.ticket = (uint64_t)i;
    q.status = make_request(problems[i], results ? &results[i] : nullptr, q);
    if (q.status == MP_OK) pending.push_back(&q);
  }
  CtxPool pool(ctx);
  {
    Engine<float> ef(ctx, &pool, cs);
    Engine<double> ed(ctx, &pool, cs);
    bool broken = false;
    int64_t escalations = 0;
    while (!broken && (!pending.empty() || !ef.idle() || !ed.idle())) {
      while (!pending.empty()) {
        Request* q = pending.front();
        const bool idle = ef.idle() && ed.idle();
        mp_status a = q->precision == 0 ? ed.admit(q) : ef.admit(q);
        if (a == MP_E_OOM && !idle) break;  // retry once resident cells finish
        pending.pop_front();
        if (a != MP_OK) {
          q->status = a;
          if (q->message.empty()) q->message = "device memory exhausted for this cell";
        }
      }
      std::vector<Request*> fin;
      if (ef.round(fin) == MP_E_CUDA || ed.round(fin) == MP_E_CUDA) broken = true;
      if (!broken) {
        escalations += migrate(ef, ed);
        migrate(ed, ef);
      }
    }
    if (stats) {
      stats->rounds = ef.rounds();
      stats->rounds_fp64 = ed.rounds();
      stats->voxel_iters = ef.voxel_iters() + ed.voxel_iters();
      stats->voxel_iters_fp64 = ed.voxel_iters();
      stats->escalations = escalations;
      stats->delta_switches = ef.delta_switches();
    }
    for (Request* q : pending) {
      q->status = MP_E_CUDA;
      q->message = "not run: an earlier batched round failed on the device";
    }
  }
  mp_status overall = MP_OK;
  for (int i = 0; i < count; ++i) {
    if (per_item) per_item[i] = reqs[i].status;
    if (reqs[i].status != MP_OK && overall == MP_OK) {
      overall = reqs[i].status;
      set_error(ctx, overall, "item %d: %s", i, reqs[i].message.c_str());
    }
  }
  return overall;
}

mp_status mp_server_create(mp_ctx* ctx, const mp_server_opts* opts, mp_server** out) {
  if (!ctx || !out) return set_error(nullptr, MP_E_INVALID_ARG, "NULL argument");
  *out = nullptr;
  MP_DEVICE_SCOPE(ctx);
  mp_status st = MP_OK;
  size_t budget = opts ? opts->hbm_budget_bytes : 0;
  if (budget == 0) {
    size_t free_b = 0, total_b = 0;
    MP_CK(ctx, cudaMemGetInfo(&free_b, &total_b));
    budget = free_b / 2;
  }
  budget = budget / kAlign * kAlign;
  if (budget < (1u << 20)) return set_error(ctx, MP_E_INVALID_ARG, "HBM budget below 1 MiB");
  mp_server* S = new mp_server();
  S->ctx = ctx;
  S->wctx.device = ctx->device;
  S->wctx.nsm = ctx->nsm;
  S->max_resident = (opts && opts->max_resident > 0) ? opts->max_resident : 1024;
  if ((st = dalloc(ctx, S->block, budget)) != MP_OK) {
    delete S;
    return st;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    dfree(ctx, S->block);
    delete S;
    return set_error(ctx, MP_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
  }
  S->pool = new BlockPool(S->block.ptr, S->block.bytes);
  S->ef = new Engine<float>(&S->wctx, S->pool, S->stream);
  S->ed = new Engine<double>(&S->wctx, S->pool, S->stream);
  S->worker = std::thread(server_loop, S);
  *out = S;
  return MP_OK;
}

mp_status mp_server_submit(mp_server* S, const mp_problem* problem, mp_result* result, uint64_t* ticket) {
  if (!S || !ticket) return set_error(nullptr, MP_E_INVALID_ARG, "NULL argument");
  *ticket = 0;
  Request* q = new Request();
  mp_status st = make_request(problem, result, *q);
  if (st != MP_OK) {
    set_error(nullptr, st, "%s", q->message.c_str());
    delete q;
    return st;
  }
  if (cudaSetDevice(S->wctx.device) != cudaSuccess) {
    delete q;
    return set_error(nullptr, MP_E_NO_DEVICE, "cannot select the server's device");
  }
  q->footprint = q->precision == 0 ? S->ed->footprint(*q) : S->ef->footprint(*q);
  if (q->footprint > S->block.bytes) {
    const size_t need = q->footprint;
    delete q;
    return set_error(nullptr, MP_E_OOM, "request needs %zu device bytes, above the server's budget of %zu", need,
                     S->block.bytes);
  }
  q->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete q;
      return set_error(nullptr, MP_E_CANCELLED, "server is shutting down");
    }
    q->ticket = S->next_ticket++;
    S->reqs[q->ticket] = q;
    S->queue.push_back(q);
    S->submitted++;
    *ticket = q->ticket;
  }
  S->cv_work.notify_one();
  return MP_OK;
}

mp_status mp_server_wait(mp_server* S, uint64_t ticket, int32_t timeout_ms) {
  if (!S) return set_error(nullptr, MP_E_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return set_error(nullptr, MP_E_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  Request* q = it->second;
  auto ready = [&] { return q->done; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return set_error(nullptr, MP_E_TIMEOUT, "ticket %llu not finished within %d ms", (unsigned long long)ticket,
                     timeout_ms);
  }
  const mp_status st = q->status;
  if (st != MP_OK) set_error(nullptr, st, "%s", q->message.c_str());
  S->reqs.erase(it);
  delete q;
  return st;
}

mp_status mp_server_query(mp_server* S, mp_server_stats* out) {
  if (!S || !out) return set_error(nullptr, MP_E_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->queued = (int64_t)S->queue.size();
  out->resident = S->resident;
  out->peak_resident = S->peak_resident;
  out->rounds = S->rounds;
  out->voxel_iters = S->voxel_iters;
  out->budget_bytes = S->block.bytes;
  out->resident_bytes = S->resident_bytes;
  return MP_OK;
}

void mp_server_destroy(mp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->wctx.device);
  delete S->ef;
  delete S->ed;
  delete S->pool;
  for (auto& kv : S->reqs) delete kv.second;
  S->reqs.clear();
  if (S->stream) cudaStreamDestroy(S->stream);
  dfree(S->ctx, S->block);
  delete S;
}

}  // extern "C"
