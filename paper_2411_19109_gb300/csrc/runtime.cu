// Host runtime and C ABI of the LLG solver (declared in include/llg.h).
//
// A context owns, for a batch of instances packed back to back:
//   * the instance descriptors and the row / column work-tile tables that
//     let every kernel launch cover the whole batch (uneven grid sizes);
//   * one demag spectrum table per distinct grid shape, built in FP64;
//   * the forward state (m, two stage buffers, RK accumulator), the demag
//     spectrum pool, the periodic checkpoints and one recorded segment
//     (stage inputs Y_s and fields B_s of up to K steps), and the adjoint
//     state (lambda, stage sums, Bbar ping-pong, Kahan pair for dJ/dpsi);
//   * the checkpoint action list it executes.
// Checkpointing follows the paper's memory argument (Introduction and the
// adjoint-state section): only every K-th state is kept and each segment is
// recomputed once during the reverse sweep, O(sqrt N) states at the default K;
// or binomial checkpointing with a fixed number of snapshot slots, which
// trades more recomputation for memory independent of the segment length.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "llg.h"
#include "regfft.cuh"
#include "dopri.cuh"

using namespace llg;

namespace {

enum Op { SNAP = 0, ADVANCE = 1, RESTORE = 2, RECORD = 3, REVERSE = 4 };
struct Action { long long op, a, b; };

long long isqrt_ceil(long long n) {
  if (n <= 0) return 1;
  long long k = (long long)std::sqrt((double)n);
  while (k * k > n) --k;
  while (k * k < n) ++k;
  return k;
}

// C(s + r, s), saturated at 2^62.
long long binom_sat(long long s, long long r) {
  const long long cap = 1LL << 62;
  const long long k = std::min(s, r), base = s + r - k;
  long long v = 1;
  for (long long j = 1; j <= k; ++j) {
    const __int128 w = (__int128)v * (base + j) / j;
    if (w >= cap) return cap;
    v = (long long)w;
  }
  return v;
}

// Binomial schedule with s free snapshot slots (slot 0 holds m_0).  Reversing
// l steps from a snapshot at a with s free slots, each step advanced at most r
// times, works exactly when l <= C(s + r, s): take the smallest such r, put
// right = min(C(s - 1 + r, s - 1), l - 1) steps after the split, advance to
// the split and snapshot there, reverse the right part with s - 1 slots, then
// the left part with s.  With no free slot, re-advance from a for every step.
// Each step is recorded singly just before it is reversed.  The first descent
// (advance, snapshot, ..., record the last step) is the forward pass.
void make_binomial(long long N, long long s0, std::vector<Action>& fwd, std::vector<Action>& rev) {
  std::vector<Action> out;
  out.push_back({SNAP, 0, 0});
  long long cur = 0;   // step the working state holds with a valid spectrum, -1 if none
  auto go = [&](long long a, long long slot) {
    if (cur != a) {
      out.push_back({RESTORE, slot, a});
      cur = a;
    }
  };
  auto rec_rev = [&](long long n) {
    out.push_back({RECORD, n, n + 1});
    out.push_back({REVERSE, n + 1, n});
    cur = -1;
  };
  struct Task { long long a, len, s, slot; };
  std::vector<Task> tasks{{0, N, s0, 0}};
  while (!tasks.empty()) {
    const Task t = tasks.back();
    tasks.pop_back();
    if (t.len == 1) {
      go(t.a, t.slot);
      rec_rev(t.a);
    } else if (t.s == 0) {
      for (long long k = t.len - 1; k >= 0; --k) {
        go(t.a, t.slot);
        if (k > 0) {
          out.push_back({ADVANCE, t.a, t.a + k});
          cur = t.a + k;
        }
        rec_rev(t.a + k);
      }
    } else {
      long long r = 1;
      while (binom_sat(t.s, r) < t.len) ++r;
      const long long right = std::min(binom_sat(t.s - 1, r), t.len - 1);
      const long long mid = t.a + t.len - right;
      go(t.a, t.slot);
      out.push_back({ADVANCE, t.a, mid});
      cur = mid;
      out.push_back({SNAP, mid, t.slot + 1});
      tasks.push_back({t.a, t.len - right, t.s, t.slot});
      tasks.push_back({mid, right, t.s - 1, t.slot + 1});
    }
  }
  size_t first = 0;
  while (out[first].op != RECORD) ++first;
  fwd.assign(out.begin(), out.begin() + first + 1);
  rev.assign(out.begin() + first + 1, out.end());
}

// Periodic schedule: snapshots at n = 0, K, 2K, ..; the forward records the
// last segment; the reverse restores, re-records and reverses each earlier
// segment.  Store-all is the same schedule with K = 1 (every state kept).
void make_schedule(long long N, int ckpt, int seg_len, std::vector<Action>& fwd, std::vector<Action>& rev) {
  fwd.clear();
  rev.clear();
  if (N <= 0) return;
  if (ckpt == LLG_CKPT_BINOMIAL) {
    make_binomial(N, seg_len > 0 ? seg_len : isqrt_ceil(N), fwd, rev);
    return;
  }
  long long K = (ckpt == LLG_CKPT_STORE_ALL) ? 1 : (seg_len > 0 ? seg_len : isqrt_ceil(N));
  const long long nseg = (N + K - 1) / K;
  for (long long c = 0; c < nseg; ++c) {
    const long long a = c * K, b = std::min(N, (c + 1) * K);
    if (c + 1 < nseg) {
      fwd.push_back({SNAP, a, c});
      fwd.push_back({ADVANCE, a, b});
    } else {
      fwd.push_back({RECORD, a, b});
    }
  }
  for (long long c = nseg - 1; c >= 0; --c) {
    const long long a = c * K, b = std::min(N, (c + 1) * K);
    if (c + 1 < nseg) {
      rev.push_back({RESTORE, c, a});
      rev.push_back({RECORD, a, b});
    }
    rev.push_back({REVERSE, b, a});
  }
}

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Launch configurations chosen by timing (LLG_TUNE_MEASURE), per process,
// keyed by device, precision, adjoint spectrum and the batch's grid shapes.
std::mutex g_tune_mutex;
std::map<std::string, llg_launch> g_tune_cache;
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

struct llg_ctx {
  std::string err;
  virtual ~llg_ctx() {}
  virtual llg_status forward(const void* phi, const void* m0, double* J, void* mT) = 0;
  virtual llg_status adjoint(const double* wext, void* dphi, void* dm0) = 0;
  virtual llg_status adaptive_steps(int inst, double* t, double* h, long long cap, long long* count) = 0;
  virtual llg_status levelset(void* phi, const void* grad, const unsigned char* mask, double lr) = 0;
  virtual llg_status field(const void* phi, const void* m, double t, int demag_only, void* B) = 0;
  virtual size_t device_bytes() const = 0;
  virtual double last_ms() const = 0;
  virtual long long launches() const = 0;
  virtual void kernel_time(int family, long long* count, double* ms) = 0;
  llg_launch L{16, 2, 2, 2, 1};   // the launch configuration in use
  double tune_ms = 0.0;        // host time spent timing candidates at create
};

template <typename T>
struct Engine final : llg_ctx {
  using C = cplx<T>;
  std::vector<llg_problem> P;
  int n = 0;
  llg_options opt{};
  cudaStream_t st = nullptr;
  long long N = 0, n_from = 0;
  double dt = 0;

  std::vector<DevInst> H;
  std::vector<RowTile> rt;
  // column tiles of films (8- and 16-element FFT lanes) and of 3D grids
  std::vector<ColTile> ct, ct16, ct3;
  DevInst* dI = nullptr;
  RowTile* dRT = nullptr;
  // row tiles of films and of 3D grids (the row-family and adjoint kernels
  // have a variant for each; the elementwise kernels take all tiles)
  std::vector<RowTile> rt2, rt3;
  RowTile *dRT2 = nullptr, *dRT3 = nullptr;
  ColTile* dCT = nullptr;
  ColTile* dCT3 = nullptr;
  ColTile* dCT16 = nullptr;
  int R = 2, TX = 8;
  size_t smem = 0, smem_rows = 0, smem_cols = 0, smem_c3 = 0, smem_adj = 0, smem_misc = 0;
  int* errw = nullptr;
  long long total_nodes = 0, total_spec = 0, total_tens = 0;
  long long K = 1, nckpt = 0, rec_steps = 0;
  std::vector<Action> fwd, rev;

  T *psi = nullptr, *dpsi = nullptr, *m = nullptr, *Ya = nullptr, *Yb = nullptr, *acc = nullptr;
  T *tens = nullptr, *recY = nullptr, *recB = nullptr, *ckpt = nullptr;
  T *lam = nullptr, *G = nullptr, *gpart = nullptr, *bb[2] = {nullptr, nullptr};
  T *psib = nullptr, *psic = nullptr;
  C *spec = nullptr, *tw = nullptr;
  double2* tw64 = nullptr;
  // double-float frequency domain of the adjoint's demag transpose (FP32
  // contexts with llg_options.adj_spectral = LLG_SPEC_DFLOAT): its own
  // spectrum pool, twiddle table and tensor tables (hi + lo pairs of the
  // FP64-built spectra)
  bool adj_df = false;
  dcplx *spec_df = nullptr, *tw_df = nullptr;
  dfloat* tens_df = nullptr;
  size_t smem_cols_df = 0, smem_adj_df = 0;
  // split double-float adjoint stage (llg_launch.adj_split): the node
  // phase's FP32 kernel and the double-float row transforms, which pass the
  // demag transpose through Dbuf (3 x nodes)
  T* Dbuf = nullptr;
  size_t smem_split = 0, smem_rows_df = 0;
  // per-(step, row tile) objective partials, per-row-tile terminal and psi
  // partials, per-instance J
  double *slots = nullptr, *jterm = nullptr, *psitile = nullptr, *Jd = nullptr, *rf = nullptr;
  // spectral objective: port partials per (step, tile, box), port series and
  // per-step adjoint weights per (instance, step, box), host copies
  double *pslots = nullptr, *Pd = nullptr, *wtab = nullptr;
  bool any_spec = false;   // an instance with the spectral or the curve objective
  std::vector<double> hP, hW, Jspec;
  // per instance: the tabulated drive (empty: sine) and the curve samples,
  // copied at create (the caller's arrays need not outlive llg_create)
  std::vector<std::vector<double>> drive_tab;
  struct CurveSamples {
    std::vector<long long> step;
    std::vector<double> target, weight;
  };
  std::vector<CurveSamples> curve;
  double* psimom = nullptr;   // per row tile: sum psi x, sum psi y
  // Dormand-Prince integrator: slopes k_1..k_7, the fifth-order solution,
  // store-all checkpoints of the accepted steps, the reverse sweep's stage
  // record and eta slots, per-tile error sums, per-instance step state
  // (t, h, last, done), acceptance, accepted-step counts and schedule
  bool dp_mode = false;
  long long dp_maxK = 0;
  T *dp_k = nullptr, *dp_y5 = nullptr, *dp_ck = nullptr, *dp_recY = nullptr, *dp_recB = nullptr;
  T *dp_eta = nullptr, *dp_mrev = nullptr;
  // periodic checkpoints of the accepted steps (LLG_CKPT_PERIODIC): m every
  // dp_K-th accepted step; the reverse sweep replays each block's steps from
  // the recorded (t, h) into dp_seg (up to 2 dp_K states) before reversing
  // them.  dp_K = 1: one checkpoint per accepted step, no replay.
  long long dp_K = 1;
  T* dp_seg = nullptr;
  long long *dp_k0 = nullptr, *dp_khi = nullptr, *dp_ckslot = nullptr;
  double *dp_e = nullptr, *dp_hst = nullptr, *dp_sched = nullptr;
  int *dp_acc = nullptr, *dp_cnt = nullptr, *dp_ovf = nullptr;
  long long* dp_slot = nullptr;
  std::vector<int> dp_cnt_h;
  long long total_slots = 0;
  long long* step_base = nullptr;
  unsigned int* maxbits = nullptr;
  double* wext = nullptr;   // per-instance cotangents of J (llg_adjoint's dJ_dextra)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  double ms = 0.0;
  long long nlaunch = 0;
  bool have_fwd = false;
  const T* mN_ptr = nullptr;

  // CUDA graphs of whole segments, keyed by (segment kind, length).  A
  // segment's launches depend only on its kind and length (the first step
  // number is read from *step_base), so one capture serves every segment of
  // that shape.  Value: the executable graph and the launches it holds.
  // ADVANCE_ADJ: recomputation during the reverse sweep (no objective terms).
  // The cache holds at most kMaxGraphs graphs; other shapes run directly.
  enum SegKind { SEG_ADVANCE = 0, SEG_RECORD_FWD = 1, SEG_RECORD_ADJ = 2, SEG_REVERSE = 3, SEG_ADVANCE_ADJ = 4,
                 SEG_DP_ATTEMPT = 5, SEG_DP_REVERSE = 6, SEG_DP_REPLAY = 7 };
  static constexpr size_t kMaxGraphs = 64;
  std::map<std::pair<int, long long>, std::pair<cudaGraphExec_t, long long>> graphs;
  cudaStream_t cap_st = nullptr;   // private stream the captures are recorded on
  // Two instance groups (even and odd index) whose RK4 segments run as two
  // independent chains on two streams (two branches of each captured graph),
  // so that one group's launches fill the other's last wave and kernels of
  // different kinds share the SMs.  Each tile list has a partitioned device
  // copy (group 0's tiles first); grp_sel selects the part the launch helpers
  // take (-1: the whole list in its original order, which measured faster
  // for single launches).
  bool two_groups = false;
  int grp_sel = -1;
  size_t split_rt2 = 0, split_rt3 = 0, split_ct = 0, split_ct16 = 0, split_ct3 = 0;
  RowTile *dRT2p = nullptr, *dRT3p = nullptr;
  ColTile *dCTp = nullptr, *dCT16p = nullptr, *dCT3p = nullptr;
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // (offset, count) of the selected group in a tile list of size sz split at sp
  std::pair<size_t, size_t> part(size_t sz, size_t sp) const {
    if (grp_sel < 0) return {0, sz};
    return grp_sel == 0 ? std::make_pair((size_t)0, sp) : std::make_pair(sp, sz - sp);
  }

  ~Engine() override {
    if (st) cudaStreamSynchronize(st);
    for (auto& g : graphs) cudaGraphExecDestroy(g.second.first);
    if (cap_st) cudaStreamDestroy(cap_st);
    if (st2) cudaStreamDestroy(st2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    for (void* p : allocs) cudaFree(p);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (Timer& tm : timers)
      for (cudaEvent_t e : tm.ev) cudaEventDestroy(e);
  }

  size_t device_bytes() const override { return bytes; }
  double last_ms() const override { return ms; }
  long long launches() const override { return nlaunch; }

  // per-family event timing: pairs recorded around launches, drained after
  // every synchronising API call
  struct Timer {
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    long long count = 0;
    double ms = 0.0;
  };
  Timer timers[5];
  void time_begin(int fam) {
    if (!opt.time_kernels) return;
    Timer& tm = timers[fam];
    if (tm.used + 2 > tm.ev.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      tm.ev.push_back(a);
      tm.ev.push_back(b);
    }
    cudaEventRecord(tm.ev[tm.used], st);
  }
  void time_end(int fam) {
    if (!opt.time_kernels) return;
    Timer& tm = timers[fam];
    cudaEventRecord(tm.ev[tm.used + 1], st);
    tm.used += 2;
  }
  void time_drain() {
    for (Timer& tm : timers) {
      for (size_t i = 0; i + 1 < tm.used; i += 2) {
        float f = 0.f;
        if (cudaEventElapsedTime(&f, tm.ev[i], tm.ev[i + 1]) == cudaSuccess) {
          tm.ms += f;
          tm.count += 1;
        }
      }
      tm.used = 0;
    }
  }
  void kernel_time(int family, long long* count, double* ms) override {
    if (family < 0 || family > 4) {
      if (count) *count = 0;
      if (ms) *ms = 0.0;
      return;
    }
    if (count) *count = timers[family].count;
    if (ms) *ms = timers[family].ms;
  }

  llg_status fail(llg_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  llg_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return LLG_ECUDA;
  }

  template <typename P_>
  bool alloc(P_** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&q, count * sizeof(P_)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(q);
    bytes += count * sizeof(P_);
    *p = static_cast<P_*>(q);
    return true;
  }

  size_t slot() const { return (size_t)3 * total_nodes; }
  T* recY_slot(long long i) { return recY + (size_t)i * slot(); }
  T* recB_slot(long long i) { return recB + (size_t)i * slot(); }
  // The segment record.  LLG_RECORD_STAGES: every step's four stage inputs
  // Y_s (Y_1 = m_l) and fields B_s, recorded once by the RECORD segment.
  // LLG_RECORD_STATES: only m_l per step; each reverse step recomputes its
  // stages into one of two step records (parity of l), because adjoint
  // stage 1 of step l already needs stage 4 of step l - 1.
  bool rec_states = false;
  T* mtmp = nullptr;          // states: m_{l+1} of a recomputed step (not kept)
  C* spec2 = nullptr;         // states: the recomputation's own spectrum pool
  T* Mrec(long long l) { return rec_states ? recY_slot(l) : recY_slot(4 * l); }
  T* Yrec(long long l, int s) {
    if (!rec_states) return recY_slot(4 * l + s - 1);
    return s == 1 ? Mrec(l) : recB_slot(7 * (l & 1) + s - 2);
  }
  T* Brec(long long l, int s) {
    if (!rec_states) return recB_slot(4 * l + s - 1);
    return recB_slot(7 * (l & 1) + 3 + s - 1);
  }

  // ---------------------------------------------------------------- create
  llg_status create(const llg_problem* probs, int n_inst, const llg_options* o, cudaStream_t stream) {
    n = n_inst;
    st = stream;
    opt = *o;
    P.assign(probs, probs + n_inst);
    if (opt.integrator != LLG_INT_RK4 && opt.integrator != LLG_INT_DOPRI5) return fail(LLG_EINVAL, "unknown integrator");
    dp_mode = opt.integrator == LLG_INT_DOPRI5;
    if (dp_mode) {
      if (!(opt.rtol > 0 && opt.atol > 0 && std::isfinite(opt.rtol) && std::isfinite(opt.atol)))
        return fail(LLG_EINVAL, "the adaptive integrator needs finite rtol > 0 and atol > 0");
      for (int i = 0; i < n_inst; ++i)
        if (probs[i].objective != LLG_J_ENERGY_AREA || probs[i].drive)
          return fail(LLG_EINVAL, "the adaptive integrator needs the LLG_J_ENERGY_AREA objective and the sine drive");
    }
    N = P[0].nsteps;
    n_from = P[0].n_from;
    dt = P[0].dt;
    for (int i = 0; i < n; ++i) {
      const llg_problem& p = P[i];
      char buf[256];
      if (p.nx < 4 || p.nx % 4 != 0 || p.nx > kMaxLx) {
        snprintf(buf, sizeof buf, "instance %d: nx=%d must be a multiple of 4 in [4, %d]", i, p.nx, kMaxLx);
        return fail(LLG_EINVAL, buf);
      }
      if (p.ny < 1 || p.ny > kMaxPy / 2) {
        snprintf(buf, sizeof buf, "instance %d: ny=%d must be in [1, %d]", i, p.ny, kMaxPy / 2);
        return fail(LLG_EINVAL, buf);
      }
      if (p.nz < 1 || p.nz > kMaxNz) {
        snprintf(buf, sizeof buf, "instance %d: nz=%d must be in [1, %d]", i, p.nz, kMaxNz);
        return fail(LLG_EINVAL, buf);
      }
      if (!(p.dx > 0 && p.dy > 0 && p.dz > 0 && p.Ms > 0 && p.dt > 0 && p.A >= 0))
        return fail(LLG_EINVAL, "dx, dy, dz, Ms, dt must be > 0 and A >= 0");
      if (p.nsteps < 0 || p.nsteps != N || p.n_from != n_from || p.dt != dt)
        return fail(LLG_EINVAL, "all instances must share nsteps >= 0, n_from and dt");
      if (p.objective != LLG_J_PORT && p.objective != LLG_J_ENERGY_AREA && p.objective != LLG_J_SPECTRAL &&
          p.objective != LLG_J_CURVE)
        return fail(LLG_EINVAL, "unknown objective");
      if (p.objective == LLG_J_CURVE) {
        if (p.nsample < 1 || !p.sample_step || !p.sample_target || !p.sample_weight || p.comp < 0 || p.comp > 2)
          return fail(LLG_EINVAL, "curve objective needs nsample >= 1, the three sample arrays and comp in 0..2");
        for (int j = 0; j < p.nsample; ++j) {
          if (p.sample_step[j] < 1 || p.sample_step[j] > p.nsteps || (j > 0 && p.sample_step[j] <= p.sample_step[j - 1]))
            return fail(LLG_EINVAL, "curve objective: sample steps must increase strictly within 1..nsteps");
          if (!std::isfinite(p.sample_target[j]) || !std::isfinite(p.sample_weight[j]))
            return fail(LLG_EINVAL, "curve objective: targets and weights must be finite");
        }
        if (!std::isfinite(p.centre_w) || !std::isfinite(p.centre_target[0]) || !std::isfinite(p.centre_target[1]) ||
            !std::isfinite(p.penalty_w) || !std::isfinite(p.area_target))
          return fail(LLG_EINVAL, "curve objective: penalty weights and targets must be finite");
        any_spec = true;
      }
      if (p.drive && p.nsteps > 0)
        for (long long k = 0; k < 3 * p.nsteps + 3; ++k)
          if (!std::isfinite(p.drive[k])) return fail(LLG_EINVAL, "drive table values must be finite");
      if (p.objective == LLG_J_SPECTRAL) {
        if (p.nfreq < 1 || p.nfreq > 8 || p.n_from < 1 || p.comp < 0 || p.comp > 2)
          return fail(LLG_EINVAL, "spectral objective needs 1 <= nfreq <= 8, n_from >= 1 and comp in 0..2");
        for (int q = 0; q < p.nfreq; ++q)
          if (!std::isfinite(p.freqs[q])) return fail(LLG_EINVAL, "spectral objective: frequencies must be finite");
        any_spec = true;
      }
      if (p.objective == LLG_J_PORT && (p.comp < 0 || p.comp > 2 || (p.power != 1 && p.power != 2)))
        return fail(LLG_EINVAL, "port objective needs comp in 0..2 and power 1 or 2");
      if (p.absorb_nodes < 0) return fail(LLG_EINVAL, "absorb_nodes must be >= 0");
    }
    if (opt.precision != LLG_FP32 && opt.precision != LLG_FP64)
      return fail(LLG_EINVAL, "precision must be LLG_FP32 or LLG_FP64");
    if (opt.ckpt != LLG_CKPT_PERIODIC && opt.ckpt != LLG_CKPT_STORE_ALL && opt.ckpt != LLG_CKPT_BINOMIAL)
      return fail(LLG_EINVAL, "ckpt must be LLG_CKPT_PERIODIC, LLG_CKPT_STORE_ALL or LLG_CKPT_BINOMIAL");
    if (opt.seg_len < 0) return fail(LLG_EINVAL, "seg_len must be >= 0");
    if (opt.adj_spectral != LLG_SPEC_WORKING && opt.adj_spectral != LLG_SPEC_DFLOAT)
      return fail(LLG_EINVAL, "adj_spectral must be LLG_SPEC_WORKING or LLG_SPEC_DFLOAT");
    adj_df = opt.adj_spectral == LLG_SPEC_DFLOAT;
    if (opt.record != LLG_RECORD_STAGES && opt.record != LLG_RECORD_STATES)
      return fail(LLG_EINVAL, "record must be LLG_RECORD_STAGES or LLG_RECORD_STATES");
    rec_states = opt.record == LLG_RECORD_STATES && !dp_mode;
    if (opt.tune != LLG_TUNE_DEFAULT && opt.tune != LLG_TUNE_MEASURE && opt.tune != LLG_TUNE_GIVEN)
      return fail(LLG_EINVAL, "tune must be LLG_TUNE_DEFAULT, LLG_TUNE_MEASURE or LLG_TUNE_GIVEN");
    if (opt.tune == LLG_TUNE_GIVEN) {
      const llg_launch& g = opt.launch;
      if ((g.col_lanes != 8 && g.col_lanes != 16) || (g.col_blocks != 1 && g.col_blocks != 2) ||
          (g.adj_blocks < 1 || g.adj_blocks > 3) || (g.groups != 1 && g.groups != 2) ||
          (g.adj_split != 0 && g.adj_split != 1))
        return fail(LLG_EINVAL, "launch: col_lanes 8 or 16, col_blocks and groups 1 or 2, adj_blocks 1 to 3, "
                                "adj_split 0 or 1");
      L = g;
    }
    if (adj_df) {
      if (!std::is_same<T, float>::value)
        return fail(LLG_EINVAL, "the double-float adjoint spectrum is an option of LLG_FP32 contexts");
      if (dp_mode) return fail(LLG_EINVAL, "the double-float adjoint spectrum applies to the RK4 adjoint");
      for (int i = 0; i < n_inst; ++i)
        if (probs[i].nz != 1) return fail(LLG_EINVAL, "the double-float adjoint spectrum supports films (nz = 1)");
    }

    // Tile shapes follow from the register FFTs: one component of a row FFT
    // of length Lx takes Lx/8 threads, so a 384-thread block covers 1024/Lx
    // rows; a column FFT of length Py takes Py/8 threads per component, so a
    // block covers 1024/Py columns.  FFT exchange scratch: kExch complex.
    R = 64;
    TX = 0;
    smem_cols = smem_misc = smem_rows = smem_adj = 0;
    for (int i = 0; i < n; ++i) {
      const int Lx = std::max(16, next_pow2(2 * P[i].nx)) / 2;
      const int Py = std::max(8, next_pow2(2 * P[i].ny));
      if (P[i].nz > 1)
        smem_c3 = std::max(smem_c3, cols3_smem_bytes<T>(Py, P[i].nz, cols3_per_tile(Py, P[i].nz, Lx)));
      else
        smem_cols = std::max(smem_cols, cols_smem_bytes<T>(Py));
      smem_misc = std::max(smem_misc, (size_t)(kExch + 2 * Lx) * sizeof(C));
      smem_rows = std::max(smem_rows, stage_smem_bytes<T>(Lx, P[i].nx));
      smem_adj = std::max(smem_adj, adj_smem_bytes<T>(Lx, P[i].nx));
      if (adj_df) {
        smem_cols_df = std::max(smem_cols_df, cols_smem_bytes<dfloat>(Py));
        smem_adj_df = std::max(smem_adj_df, adj_smem_bytes<float, dfloat>(Lx, P[i].nx));
        smem_split = std::max(smem_split, adj_split_smem_bytes<T>(Lx, P[i].nx));
        smem_rows_df = std::max(smem_rows_df, spec_rows_smem_bytes<dfloat>(Lx));
      }
    }
    if (std::max(smem_cols_df, smem_adj_df) > 220 * 1024)
      return fail(LLG_EINVAL, "a double-float adjoint tile does not fit in shared memory");
    smem = std::max(std::max(smem_rows, smem_adj), std::max(std::max(smem_cols, smem_c3), smem_misc));
    if (std::max(smem_rows, smem_adj) > 220 * 1024)
      return fail(LLG_EINVAL, "a row tile does not fit in shared memory (nx too large for this precision: the "
                              "adjoint stages 7 node arrays over 3 rows; FP64 takes nx <= 780)");
    if (smem > 220 * 1024)
      return fail(LLG_EINVAL, "a column tile does not fit in shared memory (3D: nz * 2ny too large for "
                              "this precision)");
    // descriptors, shapes, tiles
    struct Shape { int nx, ny, nz; double dx, dy, dz; long long off; int Px, Py, Pz; };
    std::vector<Shape> shapes;
    H.resize(n);
    drive_tab.assign(n, {});
    curve.assign(n, {});
    for (int i = 0; i < n; ++i) {
      llg_problem& p = P[i];
      if (p.drive && N > 0) drive_tab[i].assign(p.drive, p.drive + 3 * N + 3);
      if (p.objective == LLG_J_CURVE) {
        curve[i].step.assign(p.sample_step, p.sample_step + p.nsample);
        curve[i].target.assign(p.sample_target, p.sample_target + p.nsample);
        curve[i].weight.assign(p.sample_weight, p.sample_weight + p.nsample);
      }
      p.drive = nullptr;   // the caller's arrays are not kept
      p.sample_step = nullptr;
      p.sample_target = nullptr;
      p.sample_weight = nullptr;
    }
    long long node_off = 0, spec_off = 0, tens_off = 0;
    for (int i = 0; i < n; ++i) {
      const llg_problem& p = P[i];
      DevInst d;
      std::memset(&d, 0, sizeof d);
      d.nx = p.nx; d.ny = p.ny; d.nz = p.nz;
      d.Pz = pz_of(p.nz);
      const int Px = std::max(16, next_pow2(2 * p.nx));
      d.Lx = Px / 2;
      d.Py = std::max(8, next_pow2(2 * p.ny));
      d.log2Lx = ilog2(d.Lx);
      d.log2Py = ilog2(d.Py);
      int sid = -1;
      for (size_t s = 0; s < shapes.size(); ++s)
        if (shapes[s].nx == p.nx && shapes[s].ny == p.ny && shapes[s].nz == p.nz && shapes[s].dx == p.dx &&
            shapes[s].dy == p.dy && shapes[s].dz == p.dz)
          sid = (int)s;
      if (sid < 0) {
        shapes.push_back({p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, tens_off, Px, d.Py, d.Pz});
        tens_off += tensor_table_len(Px, d.Py, d.Pz);
        sid = (int)shapes.size() - 1;
      }
      d.shape = sid;
      d.tens_off = shapes[sid].off;
      d.layer = (long long)p.nx * p.ny;
      d.nodes = d.layer * p.nz;
      d.node_off = node_off;
      node_off += d.nodes;
      d.spec_off = spec_off;
      spec_off += (long long)p.nz * p.ny * 3 * d.Lx;
      d.ntile = p.nz * ((p.ny + rows_per_tile(d.Lx) - 1) / rows_per_tile(d.Lx));
      d.tile_off = (int)rt.size();
      d.slot_off = total_slots;
      total_slots += (long long)d.ntile * (N + 1);
      d.rf_off = (long long)i * 3 * (N + 1);
      d.wt_off = (long long)i * 2 * (N + 1);
      d.Ms = p.Ms;
      d.cex_x = 2.0 * p.A / (p.Ms * p.dx * p.dx);
      d.cex_y = 2.0 * p.A / (p.Ms * p.dy * p.dy);
      d.cex_z = 2.0 * p.A / (p.Ms * p.dz * p.dz);
      d.kan = 2.0 * p.Ku / p.Ms;
      const double kn = std::sqrt(p.ku[0] * p.ku[0] + p.ku[1] * p.ku[1] + p.ku[2] * p.ku[2]);
      for (int c = 0; c < 3; ++c) d.ku[c] = kn > 0 ? p.ku[c] / kn : 0.0;
      d.alpha = p.alpha;
      d.alpha_edge = p.alpha_edge;
      d.absorb_nodes = p.absorb_nodes;
      d.absorb_x = p.absorb_x;
      d.absorb_y = p.absorb_y;
      for (int c = 0; c < 4; ++c) d.src[c] = p.src[c];
      for (int c = 0; c < 3; ++c) {
        d.B_bias[c] = p.B_bias[c];
        d.rf_dir[c] = p.rf_dir[c];
      }
      d.b_rf = p.b_rf;
      d.f_rf = p.f_rf;
      d.sigmoid_a = p.sigmoid_a;
      d.objective = p.objective;
      d.comp = p.comp;
      d.power = p.power;
      for (int b = 0; b < 2; ++b) {
        int x0 = std::max(0, p.boxes[b][0]), x1 = std::min(p.nx, p.boxes[b][1]);
        int y0 = std::max(0, p.boxes[b][2]), y1 = std::min(p.ny, p.boxes[b][3]);
        if (x1 < x0) x1 = x0;
        if (y1 < y0) y1 = y0;
        d.boxes[b][0] = x0; d.boxes[b][1] = x1; d.boxes[b][2] = y0; d.boxes[b][3] = y1;
        const long long cnt = (long long)(x1 - x0) * (y1 - y0) * p.nz;   // boxes span every layer
        d.wbox[b] = cnt > 0 ? p.weights[b] / (double)cnt : 0.0;
      }
      d.V = p.dx * p.dy * p.dz;
      d.ihx2 = 1.0 / (p.dx * p.dx);
      d.ihy2 = 1.0 / (p.dy * p.dy);
      d.ihz2 = 1.0 / (p.dz * p.dz);
      d.escale = 1.0 / (0.5 * kMu0 * p.Ms * p.Ms * d.V * (double)d.nodes);
      d.A = p.A;
      d.area_target = p.area_target;
      d.penalty_w = p.penalty_w;
      d.centre_w = p.objective == LLG_J_CURVE ? p.centre_w : 0.0;
      d.centre_x0 = p.centre_target[0];
      d.centre_y0 = p.centre_target[1];
      fill_coef(d);
      H[i] = d;
      const int rows = rows_per_tile(d.Lx);
      for (int z = 0, k = 0; z < p.nz; ++z)
        for (int y0 = 0; y0 < p.ny; y0 += rows, ++k) rt.push_back({i, z, y0, std::min(rows, p.ny - y0), k});
      const int tx = p.nz > 1 ? cols3_per_tile(d.Py, p.nz, d.Lx) : std::max(1, std::min(1024 / d.Py, d.Lx));
      const bool c16 = sizeof(T) == 4 && p.nz == 1 && cols16_length(d.Py);
      for (int k0 = 0; k0 < d.Lx; k0 += tx)
        (p.nz > 1 ? ct3 : (c16 ? ct16 : ct)).push_back({i, k0, std::min(tx, d.Lx - k0), 0});
      TX = std::max(TX, tx);
    }
    total_nodes = node_off;
    total_spec = spec_off;
    total_tens = tens_off;

    make_schedule(N, opt.ckpt, opt.seg_len, fwd, rev);
    K = (opt.ckpt == LLG_CKPT_STORE_ALL) ? 1 : (opt.seg_len > 0 ? opt.seg_len : isqrt_ceil(N));
    K = std::max(1LL, std::min(K, std::max(N, 1LL)));
    nckpt = 0;
    rec_steps = 0;
    for (const Action& a : fwd)
      if (a.op == SNAP) nckpt = std::max(nckpt, a.b + 1);
    for (const Action& a : fwd)
      if (a.op == RECORD) rec_steps = std::max(rec_steps, a.b - a.a);
    for (const Action& a : rev)
      if (a.op == RECORD) rec_steps = std::max(rec_steps, a.b - a.a);

    const size_t S = slot();
    for (const RowTile& t : rt) (H[t.inst].nz > 1 ? rt3 : rt2).push_back(t);
    // the partitioned tile lists exist for every batch of two or more, so
    // that the number of chains can be chosen (or timed) after set-up
    const bool can_split = n >= 2;
    bool ok = alloc(&dI, n) && alloc(&dRT, rt.size()) && alloc(&dRT2, std::max<size_t>(1, rt2.size())) &&
              alloc(&dRT3, std::max<size_t>(1, rt3.size())) && alloc(&dCT, std::max<size_t>(1, ct.size())) &&
              alloc(&dCT3, std::max<size_t>(1, ct3.size())) && alloc(&dCT16, std::max<size_t>(1, ct16.size())) && alloc(&psi, total_nodes) &&
              alloc(&dpsi, total_nodes) && alloc(&m, S) && alloc(&Ya, S) && alloc(&Yb, S) && alloc(&acc, S) &&
              alloc(&tens, total_tens) && alloc(&spec, total_spec) && alloc(&tw, kTwiddleN) &&
              alloc(&tw64, kTwiddleN) && alloc(&recY, S * (rec_states ? rec_steps + 1 : 4 * rec_steps + 1)) &&
              alloc(&recB, S * (rec_states ? 14 : std::max(1LL, 4 * rec_steps))) && alloc(&ckpt, S * std::max(1LL, nckpt)) &&
              alloc(&lam, S) && alloc(&G, S) && alloc(&gpart, S) && alloc(&bb[0], S) && alloc(&bb[1], S) &&
              alloc(&psib, total_nodes) && alloc(&psic, total_nodes) && alloc(&slots, (size_t)total_slots) &&
              alloc(&pslots, any_spec ? 2 * (size_t)total_slots : 2) && alloc(&Pd, (size_t)n * 2 * (N + 1)) &&
              alloc(&wtab, (size_t)n * 2 * (N + 1)) &&
              alloc(&jterm, rt.size()) && alloc(&psitile, rt.size()) && alloc(&psimom, 2 * rt.size()) && alloc(&Jd, n) && alloc(&step_base, 1) &&
              alloc(&maxbits, 2 * n) && alloc(&rf, (size_t)n * 3 * (N + 1)) && alloc(&errw, 1) &&
              alloc(&wext, n);
    if (!ok) return fail(LLG_ENOMEM, "device allocation failed (" + std::to_string(bytes >> 20) + " MiB so far)");
    if (adj_df && !(alloc(&spec_df, total_spec) && alloc(&tw_df, kTwiddleN) && alloc(&tens_df, total_tens) &&
                    alloc(&Dbuf, slot())))
      return fail(LLG_ENOMEM, "device allocation failed (double-float adjoint spectrum)");
    if (rec_states && !(alloc(&mtmp, S) && alloc(&spec2, total_spec)))
      return fail(LLG_ENOMEM, "device allocation failed (step records)");
    if (can_split) {
      // partitioned copies of the tile lists: even instances first
      auto even_r = [](const RowTile& t) { return t.inst % 2 == 0; };
      auto even_c = [](const ColTile& t) { return t.inst % 2 == 0; };
      std::vector<RowTile> p2 = rt2, p3 = rt3;
      std::vector<ColTile> pc = ct, p16 = ct16, pc3 = ct3;
      split_rt2 = std::stable_partition(p2.begin(), p2.end(), even_r) - p2.begin();
      split_rt3 = std::stable_partition(p3.begin(), p3.end(), even_r) - p3.begin();
      split_ct = std::stable_partition(pc.begin(), pc.end(), even_c) - pc.begin();
      split_ct16 = std::stable_partition(p16.begin(), p16.end(), even_c) - p16.begin();
      split_ct3 = std::stable_partition(pc3.begin(), pc3.end(), even_c) - pc3.begin();
      const bool ok3 = alloc(&dRT2p, std::max<size_t>(1, p2.size())) && alloc(&dRT3p, std::max<size_t>(1, p3.size())) &&
                       alloc(&dCTp, std::max<size_t>(1, pc.size())) && alloc(&dCT16p, std::max<size_t>(1, p16.size())) &&
                       alloc(&dCT3p, std::max<size_t>(1, pc3.size()));
      if (!ok3) return fail(LLG_ENOMEM, "device allocation failed (tile lists)");
      cudaError_t e2 = cudaSuccess;
      if (!p2.empty()) e2 = cudaMemcpy(dRT2p, p2.data(), sizeof(RowTile) * p2.size(), cudaMemcpyHostToDevice);
      if (e2 == cudaSuccess && !p3.empty()) e2 = cudaMemcpy(dRT3p, p3.data(), sizeof(RowTile) * p3.size(), cudaMemcpyHostToDevice);
      if (e2 == cudaSuccess && !pc.empty()) e2 = cudaMemcpy(dCTp, pc.data(), sizeof(ColTile) * pc.size(), cudaMemcpyHostToDevice);
      if (e2 == cudaSuccess && !p16.empty()) e2 = cudaMemcpy(dCT16p, p16.data(), sizeof(ColTile) * p16.size(), cudaMemcpyHostToDevice);
      if (e2 == cudaSuccess && !pc3.empty()) e2 = cudaMemcpy(dCT3p, pc3.data(), sizeof(ColTile) * pc3.size(), cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) return cuda_fail(e2, "upload tile lists");
    }
    if (dp_mode) {
      const long long K7 = 7, R6 = 6;
      dp_maxK = opt.seg_len > 0 ? std::min<long long>(opt.seg_len, N) : N;   // accepted steps at most
      dp_K = opt.ckpt == LLG_CKPT_STORE_ALL ? 1 : std::max(1LL, isqrt_ceil(dp_maxK));
      const bool ok2 = alloc(&dp_k, S * K7) && alloc(&dp_y5, S) && alloc(&dp_ck, S * (dp_maxK / dp_K + 1)) &&
                       (dp_K == 1 || (alloc(&dp_seg, S * 2 * dp_K) && alloc(&dp_k0, n) && alloc(&dp_khi, n) &&
                                      alloc(&dp_ckslot, n))) &&
                       alloc(&dp_recY, S * R6) && alloc(&dp_recB, S * R6) && alloc(&dp_eta, S * R6) &&
                       alloc(&dp_mrev, S) && alloc(&dp_e, rt.size()) && alloc(&dp_hst, 4 * (size_t)n) &&
                       alloc(&dp_sched, 2 * (size_t)n * std::max(1LL, dp_maxK)) && alloc(&dp_acc, n) &&
                       alloc(&dp_cnt, n) &&
                       alloc(&dp_ovf, 1) && alloc(&dp_slot, n);
      if (!ok2)
        return fail(LLG_ENOMEM, "device allocation failed for the adaptive integrator's checkpoints (" +
                                    std::to_string(bytes >> 20) + " MiB so far)");
    }

    cudaError_t e;
    if ((e = cudaMemcpyAsync(dI, H.data(), sizeof(DevInst) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "upload descriptors");
    if (!rt2.empty() &&
        (e = cudaMemcpyAsync(dRT2, rt2.data(), sizeof(RowTile) * rt2.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
      return cuda_fail(e, "upload row tiles");
    if (!rt3.empty() &&
        (e = cudaMemcpyAsync(dRT3, rt3.data(), sizeof(RowTile) * rt3.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
      return cuda_fail(e, "upload row tiles");
    if ((e = cudaMemcpyAsync(dRT, rt.data(), sizeof(RowTile) * rt.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return cuda_fail(e, "upload row tiles");
    if (!ct.empty() &&
        (e = cudaMemcpyAsync(dCT, ct.data(), sizeof(ColTile) * ct.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
      return cuda_fail(e, "upload column tiles");
    if (!ct3.empty() &&
        (e = cudaMemcpyAsync(dCT3, ct3.data(), sizeof(ColTile) * ct3.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
      return cuda_fail(e, "upload column tiles");
    if (!ct16.empty() &&
        (e = cudaMemcpyAsync(dCT16, ct16.data(), sizeof(ColTile) * ct16.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
      return cuda_fail(e, "upload column tiles");
    {
      std::vector<double2> h64(kTwiddleN);
      std::vector<C> hT(kTwiddleN);
      for (int k = 0; k < kTwiddleN; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)kTwiddleN;
        h64[k] = make_double2(std::cos(ang), std::sin(ang));
        hT[k].x = (T)h64[k].x;
        hT[k].y = (T)h64[k].y;
      }
      if ((e = cudaMemcpyAsync(tw64, h64.data(), sizeof(double2) * kTwiddleN, cudaMemcpyHostToDevice, st)) !=
          cudaSuccess)
        return cuda_fail(e, "upload twiddles");
      if ((e = cudaMemcpyAsync(tw, hT.data(), sizeof(C) * kTwiddleN, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload twiddles");
      std::vector<dcplx> hD(adj_df ? kTwiddleN : 0);
      for (size_t k = 0; k < hD.size(); ++k) {
        hD[k].x = dfloat(h64[k].x);
        hD[k].y = dfloat(h64[k].y);
      }
      if (adj_df &&
          (e = cudaMemcpyAsync(tw_df, hD.data(), sizeof(dcplx) * kTwiddleN, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload twiddles");
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "create");
    }
    {
      // RF drive per step and stage time t = n dt + c dt (c = 0, 1/2, 1), in FP64
      std::vector<double> h((size_t)n * 3 * (N + 1));
      for (int i = 0; i < n; ++i)
        for (long long s = 0; s <= N; ++s)
          for (int c = 0; c < 3; ++c) {
            const double t = (double)s * dt + 0.5 * c * dt;
            h[(size_t)i * 3 * (N + 1) + 3 * s + c] =
                drive_tab[i].empty() ? P[i].b_rf * std::sin(2.0 * M_PI * P[i].f_rf * t) : drive_tab[i][3 * s + c];
          }
      if ((e = cudaMemcpyAsync(rf, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess)
        return cuda_fail(e, "upload RF table");
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "create");
    }
    // demag spectra, FP64 scratch of the largest shape
    size_t gmax = 0;
    for (const Shape& s : shapes) gmax = std::max(gmax, (size_t)tensor_scratch_len(s.Px, s.Py, s.Pz));
    double2* Gs = nullptr;
    if (cudaMalloc(&Gs, gmax * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(LLG_ENOMEM, "tensor scratch allocation failed");
    }
    for (const Shape& s : shapes) {
      e = build_tensor_spectrum<T>(tens + s.off, Gs, s.nx, s.ny, s.nz, s.Px, s.Py, s.Pz, s.dx, s.dy, s.dz, tw64,
                                   st);
      nlaunch += s.Pz > 1 ? 6 : 5;
      if (e == cudaSuccess && adj_df) {
        e = build_tensor_spectrum<dfloat>(tens_df + s.off, Gs, s.nx, s.ny, s.nz, s.Px, s.Py, s.Pz, s.dx, s.dy, s.dz,
                                          tw64, st);
        nlaunch += 5;
      }
      if (e != cudaSuccess) {
        cudaFree(Gs);
        return cuda_fail(e, "demag tensor");
      }
    }
    e = cudaStreamSynchronize(st);
    cudaFree(Gs);
    if (e != cudaSuccess) return cuda_fail(e, "demag tensor");
    set_smem_limits<T>(smem_rows, smem_misc, smem_cols, smem_adj);
    if (can_split) {
      if ((e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "create the second stream");
    }
    cudaMemsetAsync(wtab, 0, sizeof(double) * n * 2 * (N + 1), st);
    smem_cols3<T>(smem_c3);
    if constexpr (sizeof(T) == 4) smem_cols16<T>(smem_cols);
    if constexpr (std::is_same<T, float>::value) {
      if (adj_df) {
        llg::smem_cols<dfloat>(smem_cols_df);
        llg::smem_adj<float, dfloat>(smem_adj_df);
        llg::smem_adj_split<float>(smem_split);
        llg::smem_spec_rows<float, dfloat>(smem_rows_df);
      }
    }
    cudaMemsetAsync(errw, 0, sizeof(int), st);
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "create");
    if (opt.tune == LLG_TUNE_MEASURE)
      if (llg_status ts = tune(shapes_key())) return ts;
    two_groups = can_split && L.groups == 2 && !opt.time_kernels;
    return LLG_OK;
  }

  // ------------------------------------------------------------ tuning
  // Cache key: device, precision, adjoint spectrum, grid shapes with counts.
  std::string shapes_key() const {
    int dev = 0;
    cudaGetDevice(&dev);
    std::map<std::vector<double>, int> cnt;
    for (const llg_problem& p : P) ++cnt[{(double)p.nx, (double)p.ny, (double)p.nz, p.dx, p.dy, p.dz}];
    std::string k = std::to_string(dev) + "/" + std::to_string(sizeof(T)) + "/" + std::to_string(adj_df ? 1 : 0);
    char buf[160];
    for (const auto& c : cnt) {
      snprintf(buf, sizeof buf, "/%gx%gx%g:%g:%g:%g*%d", c.first[0], c.first[1], c.first[2], c.first[3], c.first[4],
               c.first[5], c.second);
      k += buf;
    }
    return k;
  }
  // median device time (ms) of `reps` runs of fn on the context stream
  template <typename F>
  double time_ms(F&& fn, int reps) {
    std::vector<float> v;
    fn();   // warm-up (and module load of the variant)
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(ev0, st);
      fn();
      cudaEventRecord(ev1, st);
      cudaEventSynchronize(ev1);
      float f = 0.f;
      cudaEventElapsedTime(&f, ev0, ev1);
      v.push_back(f);
    }
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
  }
  // Coordinate search over the launch configuration on this batch: each
  // field's alternative is timed on the launches it changes (kernel
  // contents do not affect their speed; the buffers hold whatever set-up
  // left) and kept if it is faster.  One recorded RK4 step and its
  // reverse sweep serve as the workload of the chain split.
  llg_status tune(const std::string& key) {
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        L = it->second;
        return LLG_OK;
      }
    }
    if (N < 1 || dp_mode || opt.time_kernels) return LLG_OK;
    const auto t0 = std::chrono::steady_clock::now();
    // defined contents for the timed launches (set-up left them unset)
    for (T* b : {m, psi, dpsi, lam, G, gpart, bb[0], bb[1], psib, psic})
      cudaMemsetAsync(b, 0, sizeof(T) * (b == psi || b == dpsi || b == psib || b == psic ? total_nodes : slot()), st);
    const int reps = 5;
    const bool two = n >= 2;
    auto pick = [&](int* field, int alt, auto&& fn) {
      const int cur = *field;
      const double a = time_ms(fn, reps);
      *field = alt;
      const double b = time_ms(fn, reps);
      if (!(b < 0.98 * a)) *field = cur;
    };
    set_step(0);
    if (std::is_same<T, float>::value && !ct16.empty())
      pick(&L.col_lanes, L.col_lanes == 16 ? 8 : 16, [&] { cols(); });
    if (adj_df) {
      pick(&L.col_blocks, L.col_blocks == 2 ? 1 : 2, [&] { cols_df(); });
      cudaMemcpyAsync(recY_slot(0), m, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
      step(0, true, false);
      pick(&L.adj_split, L.adj_split ? 0 : 1, [&] { reverse_segment(1); });
      // the split node phase compiles for 2 or 3 blocks per SM, the fused
      // stage for 1 or 2
      if (L.adj_split) pick(&L.adj_blocks, L.adj_blocks == 3 ? 2 : 3, [&] { reverse_segment(1); });
      else pick(&L.adj_blocks, L.adj_blocks == 2 ? 1 : 2, [&] { reverse_segment(1); });
    }
    if (two) {
      two_groups = L.groups == 2;
      const int alt = L.groups == 2 ? 1 : 2;
      const double a = time_ms([&] { segment_body(SEG_RECORD_ADJ, 1); segment_body(SEG_REVERSE, 1); }, reps);
      two_groups = alt == 2;
      const double b = time_ms([&] { segment_body(SEG_RECORD_ADJ, 1); segment_body(SEG_REVERSE, 1); }, reps);
      if (b < 0.98 * a) L.groups = alt;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch configuration timing");
    int herr = 0;
    cudaMemcpy(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr) return fail(LLG_ETIMEOUT, "a bounded device wait ran out while timing launch configurations");
    tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = L;
    return LLG_OK;
  }

  // ------------------------------------------------------------- launches
  RowArgs<T> row_args() {
    RowArgs<T> a;
    std::memset(&a, 0, sizeof a);
    a.inst = dI;
    a.tiles = dRT;
    a.spec = spec;
    a.tw = tw;
    a.psi = psi;
    a.step_base = step_base;
    a.err = errw;
    a.rf = rf;
    a.rows_max = R;
    a.dt = dt;
    a.n_from = n_from;
    a.nsteps = N;
    return a;
  }
  void rows(const RowArgs<T>& a0, int mode) {
    RowArgs<T> a = a0;
    const size_t sm = (mode == ROW_STAGE || mode == ROW_DP_STAGE) ? smem_rows : smem_misc;
    if (mode == ROW_STAGE) time_begin(0);
    const auto p2 = part(rt2.size(), split_rt2), p3 = part(rt3.size(), split_rt3);
    if (p2.second) {
      a.tiles = (grp_sel < 0 ? dRT2 : dRT2p) + p2.first;
      launch_rows<T>(a, mode, (int)p2.second, sm, st, false);
      ++nlaunch;
    }
    if (p3.second) {
      a.tiles = (grp_sel < 0 ? dRT3 : dRT3p) + p3.first;
      launch_rows<T>(a, mode, (int)p3.second, sm, st, true);
      ++nlaunch;
    }
    if (mode == ROW_STAGE) time_end(0);
  }
  void cols(C* sp = nullptr) {
    ColArgs<T> c;
    c.inst = dI;
    c.tiles = dCT;
    c.spec = sp ? sp : spec;
    c.tw = tw;
    c.tens = tens;
    c.cols_max = TX;
    c.err = errw;
    time_begin(1);
    const auto pc = part(ct.size(), split_ct), p16 = part(ct16.size(), split_ct16), p3 = part(ct3.size(), split_ct3);
    if (pc.second) {
      c.tiles = (grp_sel < 0 ? dCT : dCTp) + pc.first;
      launch_cols<T>(c, (int)pc.second, smem_cols, st);
      ++nlaunch;
    }
    if constexpr (sizeof(T) == 4) {
      if (p16.second) {
        // the same tiles (1024/Py columns each) for either lane width
        c.tiles = (grp_sel < 0 ? dCT16 : dCT16p) + p16.first;
        if (L.col_lanes == 16) launch_cols16<T>(c, (int)p16.second, smem_cols, st);
        else launch_cols<T>(c, (int)p16.second, smem_cols, st);
        ++nlaunch;
      }
    }
    if (p3.second) {
      c.tiles = (grp_sel < 0 ? dCT3 : dCT3p) + p3.first;
      launch_cols3<T>(c, (int)p3.second, smem_c3, st);
      ++nlaunch;
    }
    time_end(1);
  }
  // column pass of the adjoint's double-float frequency domain: every film
  // column tile (both film tile lists; the same columns per tile) through
  // the 8-element column kernel instantiated for dfloat
  void cols_df() {
    if constexpr (std::is_same<T, float>::value) {
      ColArgs<dfloat> c;
      c.inst = dI;
      c.spec = spec_df;
      c.tw = tw_df;
      c.tens = tens_df;
      c.cols_max = TX;
      c.err = errw;
      time_begin(3);
      const auto pc = part(ct.size(), split_ct), p16 = part(ct16.size(), split_ct16);
      if (pc.second) {
        c.tiles = (grp_sel < 0 ? dCT : dCTp) + pc.first;
        launch_cols<dfloat>(c, (int)pc.second, smem_cols_df, st, L.col_blocks);
        ++nlaunch;
      }
      if (p16.second) {
        c.tiles = (grp_sel < 0 ? dCT16 : dCT16p) + p16.first;
        launch_cols<dfloat>(c, (int)p16.second, smem_cols_df, st, L.col_blocks);
        ++nlaunch;
      }
      time_end(3);
    }
  }
  void set_step(long long v) {
    launch_set_step(step_base, v, st);
    ++nlaunch;
  }
  void fft_only(const T* Y, C* sp = nullptr) {
    RowArgs<T> a = row_args();
    a.Yin = Y;
    if (sp) a.spec = sp;
    rows(a, ROW_FFT_ONLY);
  }
  void material(const T* phi) {
    launch_material_tiles<T>(dI, dRT, (int)rt.size(), phi, psi, dpsi, psitile, psimom, st);
    ++nlaunch;
  }

  // one RK4 step: record == false -> in place on m with ping-pong stage
  // buffers; record == true -> stage inputs and fields into slot l of the
  // segment record, m_{n+1} into the next record slot
  void step(int l, bool record, bool objective) {
    for (int s = 1; s <= 4; ++s) {
      cols();
      RowArgs<T> a = row_args();
      a.local_step = l;
      a.stage = s;
      a.acc = acc;
      a.slots = objective ? slots : nullptr;
      a.pslots = objective && any_spec ? pslots : nullptr;
      if (record && !rec_states) {
        a.m = Mrec(l);
        a.Yin = Yrec(l, s);
        a.Bout = Brec(l, s);
        if (s < 4) a.Yout = Yrec(l, s + 1);
        else a.mout = Mrec(l + 1);
      } else if (record) {
        // states only: the stages run on the ping-pong buffers, m_{l+1}
        // goes to the next state slot
        a.m = Mrec(l);
        a.Yin = (s == 1) ? Mrec(l) : (s == 3 ? Yb : Ya);
        if (s < 4) a.Yout = (s == 2) ? Yb : Ya;
        else a.mout = Mrec(l + 1);
      } else {
        a.m = m;
        a.Yin = (s == 1) ? m : (s == 3 ? Yb : Ya);
        if (s < 4) a.Yout = (s == 2) ? Yb : Ya;
        else a.mout = m;
      }
      rows(a, ROW_STAGE);
    }
  }

  // LLG_RECORD_STATES: recompute step l's stage inputs and fields from m_l
  // into its step record, on the recomputation's own spectrum pool (the
  // adjoint's holds a transform in flight); no objective terms
  void recompute_step(long long l) {
    fft_only(Mrec(l), spec2);
    for (int s = 1; s <= 4; ++s) {
      cols(spec2);
      RowArgs<T> a = row_args();
      a.spec = spec2;
      a.local_step = (int)l;
      a.stage = s;
      a.acc = acc;
      a.m = Mrec(l);
      a.Yin = Yrec(l, s);
      a.Bout = Brec(l, s);
      if (s < 4) a.Yout = Yrec(l, s + 1);
      else a.mout = mtmp;
      rows(a, ROW_STAGE);
    }
  }

  // one backward sweep over a recorded segment of len steps: seed with the
  // stage-4 inputs of its last step, then the 4 len adjoint stages; S is
  // the real type of the demag transpose's frequency domain
  void reverse_segment(long long len) {
    if constexpr (std::is_same<T, float>::value) {
      if (adj_df) {
        reverse_segment_t<dfloat>(len);
        return;
      }
    }
    reverse_segment_t<T>(len);
  }
  template <typename S>
  void reverse_segment_t(long long len) {
    int cur = 0;
    if (rec_states) recompute_step(len - 1);
    {
      AdjArgs<T, S> a = adj_args<S>();
      a.local_step = (int)(len - 1);
      a.stage = 4;
      a.seed_only = 1;
      a.Yprev = Yrec(len - 1, 4);
      a.Bprev = Brec(len - 1, 4);
      a.BbarOut = bb[cur];
      adj(a);
    }
    for (long long l = len - 1; l >= 0; --l) {
      for (int s = 4; s >= 1; --s) {
        // stage 1 of step l seeds step l - 1 from its stage-4 record
        if (rec_states && s == 1 && l > 0) recompute_step(l - 1);
        if constexpr (std::is_same<S, T>::value) cols();
        else cols_df();
        AdjArgs<T, S> a = adj_args<S>();
        a.local_step = (int)l;
        a.stage = s;
        a.Ys = Yrec(l, s);
        a.Bbar = bb[cur];
        a.BbarOut = bb[1 - cur];
        if (s > 1) {
          a.Yprev = Yrec(l, s - 1);
          a.Bprev = Brec(l, s - 1);
        } else if (l > 0) {
          a.Yprev = Yrec(l - 1, 4);
          a.Bprev = Brec(l - 1, 4);
          a.seed_next = 1;
        }
        adj(a);
        if (s > 1 || a.seed_next) cur ^= 1;
      }
    }
  }

  // RK4 segments with two instance groups: fork to the second stream, run
  // each group's whole segment on its own stream, join
  void segment_body(int kind, long long len) {
    if (!two_groups || kind == SEG_DP_ATTEMPT || kind == SEG_DP_REVERSE || kind == SEG_DP_REPLAY) {
      segment_body_one(kind, len);
      return;
    }
    cudaEventRecord(ev_fork, st);
    cudaStreamWaitEvent(st2, ev_fork, 0);
    const cudaStream_t s0 = st;
    for (int g = 0; g < 2; ++g) {
      grp_sel = g;
      st = g == 0 ? s0 : st2;
      segment_body_one(kind, len);
    }
    st = s0;
    grp_sel = -1;
    cudaEventRecord(ev_join, st2);
    cudaStreamWaitEvent(st, ev_join, 0);
  }

  void segment_body_one(int kind, long long len) {
    if (kind == SEG_DP_ATTEMPT) {
      for (long long l = 0; l < len; ++l) dp_attempt();
      return;
    }
    if (kind == SEG_DP_REVERSE) {
      dp_reverse_step();
      return;
    }
    if (kind == SEG_DP_REPLAY) {
      dp_replay_step();
      return;
    }
    if (kind == SEG_REVERSE) {
      reverse_segment(len);
      return;
    }
    const bool record = kind == SEG_RECORD_FWD || kind == SEG_RECORD_ADJ;
    const bool objective = kind == SEG_ADVANCE || kind == SEG_RECORD_FWD;
    for (long long l = 0; l < len; ++l) step((int)l, record, objective);
  }

  // Runs one segment whose first step number is already in *step_base:
  // directly, or by replaying (capturing on first use) its CUDA graph.
  // Graphs are not used while per-launch CUDA-event timing is on.
  llg_status run_segment(int kind, long long len) {
    if (!opt.use_graph || opt.time_kernels) {
      segment_body(kind, len);
      return LLG_OK;
    }
    const auto key = std::make_pair(kind, len);
    auto it = graphs.find(key);
    if (it == graphs.end() && graphs.size() >= kMaxGraphs) {
      segment_body(kind, len);
      return LLG_OK;
    }
    if (it == graphs.end()) {
      // capture on a private stream (the caller's may be the legacy default
      // stream, which cannot be captured); nothing runs during capture
      cudaError_t e = cudaSuccess;
      if (!cap_st && (e = cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "create capture stream");
      const long long before = nlaunch;
      if ((e = cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin graph capture");
      cudaStream_t user = st;
      st = cap_st;
      segment_body(kind, len);
      st = user;
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cap_st, &g);
      if (e != cudaSuccess) return cuda_fail(e, "end graph capture");
      cudaGraphExec_t ge = nullptr;
      e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "instantiate segment graph");
      it = graphs.emplace(key, std::make_pair(ge, nlaunch - before)).first;
      nlaunch = before;
    }
    cudaError_t e = cudaGraphLaunch(it->second.first, st);
    if (e != cudaSuccess) return cuda_fail(e, "launch segment graph");
    nlaunch += it->second.second;
    return LLG_OK;
  }

  // Spectral objective (Eq. 10 at the window's frequencies) and curve
  // objective (Eq. 8): the series of the finished forward come to the host
  // (port means P_b[n], or P[n] = sum psi m_comp / sum psi with sum psi);
  // J and the per-step adjoint weights are formed there in FP64 (a few
  // thousand numbers per instance) and go back as wtab, which the terminal
  // and adjoint kernels read.
  llg_status spectral_weights() {
    const size_t len = (size_t)n * 2 * (N + 1);
    hP.assign(len, 0.0);
    hW.assign(len, 0.0);
    Jspec.assign(n, 0.0);
    launch_port_series(dI, n, pslots, psitile, N + 1, Pd, st);
    ++nlaunch;
    cudaError_t e = cudaMemcpyAsync(hP.data(), Pd, sizeof(double) * len, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "spectral objective: port series");
    for (int i = 0; i < n; ++i) {
      const llg_problem& p = P[i];
      const double* Pi = hP.data() + (size_t)i * 2 * (N + 1);
      double* Wi = hW.data() + (size_t)i * 2 * (N + 1);
      if (p.objective == LLG_J_CURVE) {
        // J = sum_j w_j |P_j - T_j|; dJ/dm_comp = W psi / S and the explicit
        // dJ/dpsi = W (m_comp - P) / S at each sample, W = w sign(P - T)
        const CurveSamples& cs = curve[i];
        for (size_t j = 0; j < cs.step.size(); ++j) {
          const long long k = cs.step[j];
          const double Pk = Pi[2 * k], S = Pi[2 * k + 1], d = Pk - cs.target[j];
          Jspec[i] += cs.weight[j] * std::fabs(d);
          const double W = cs.weight[j] * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0));
          Wi[2 * k] = W / S;
          Wi[2 * k + 1] = W * Pk / S;
        }
        continue;
      }
      if (p.objective != LLG_J_SPECTRAL) continue;
      for (int b = 0; b < 2; ++b) {
        const DevInst& d = H[i];
        const long long cnt = (long long)(d.boxes[b][1] - d.boxes[b][0]) * (d.boxes[b][3] - d.boxes[b][2]) * d.nz;
        if (p.weights[b] == 0.0 || cnt <= 0) continue;
        for (int q = 0; q < p.nfreq; ++q) {
          double xr = 0.0, xi = 0.0;
          for (long long k = n_from; k <= N; ++k) {
            const double th = 2.0 * M_PI * p.freqs[q] * (double)k * dt;
            xr += Pi[2 * k + b] * std::cos(th);
            xi -= Pi[2 * k + b] * std::sin(th);
          }
          const double amp = std::hypot(xr, xi);
          Jspec[i] += p.weights[b] * amp;
          if (!(amp > 0.0)) continue;
          for (long long k = n_from; k <= N; ++k) {
            const double th = 2.0 * M_PI * p.freqs[q] * (double)k * dt;
            Wi[2 * k + b] += p.weights[b] * (xr * std::cos(th) - xi * std::sin(th)) / amp / (double)cnt;
          }
        }
      }
    }
    e = cudaMemcpyAsync(wtab, hW.data(), sizeof(double) * len, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "spectral objective: weights");
    return LLG_OK;
  }

  // ------------------------------------------------------------ forward
  // ------------------------------------------------ Dormand-Prince forward
  // Kernel arguments of DP stage s (1..7): the combination a(s+1, j) of the
  // next stage input, or at s = 7 the error weights b_j - b*_j.
  RowArgs<T> dp_args(int s) {
    RowArgs<T> a = row_args();
    a.hst = dp_hst;
    a.kbuf = dp_k;
    a.kstride = (long long)slot();
    a.stage = s;
    if (s < 7)
      for (int j = 1; j <= s; ++j) a.dpa[j - 1] = (T)dp::a(s + 1, j);
    else
      for (int j = 1; j <= 7; ++j) a.dpe[j - 1] = (T)dp::e(j);
    a.rtol = opt.rtol;
    a.atol = opt.atol;
    a.eslots = dp_e;
    return a;
  }
  // stage s: field and slope at Y_s (whose spectrum the last row pass left),
  // next stage input Y_{s+1} and its spectrum (s < 7)
  void dp_stage(int s, const T* Yin, const T* mm, T* Yout, T* Bout) {
    cols();
    RowArgs<T> a = dp_args(s);
    a.Yin = Yin;
    a.m = mm;
    a.Yout = Yout;
    a.Bout = Bout;
    rows(a, ROW_DP_STAGE);
  }
  // apply the controller's decision (m <- y5, k_1 <- k_7, checkpoint) and
  // form Y_2 = m + h a(2, 1) k_1 with its spectrum
  void dp_start() {
    RowArgs<T> a = row_args();
    a.hst = dp_hst;
    a.kbuf = dp_k;
    a.kstride = (long long)slot();
    a.dpa[0] = (T)dp::a(2, 1);
    a.accept = dp_acc;
    a.cnt = dp_cnt;
    a.ckall = dp_ck;
    a.ck_every = (int)dp_K;
    a.y5 = dp_y5;
    a.m = m;
    a.mout = m;
    a.Yin = m;
    a.Yout = Ya;
    rows(a, ROW_DP_START);
  }
  void dp_attempt() {
    dp_stage(2, Ya, m, Yb, nullptr);
    dp_stage(3, Yb, m, Ya, nullptr);
    dp_stage(4, Ya, m, Yb, nullptr);
    dp_stage(5, Yb, m, Ya, nullptr);
    dp_stage(6, Ya, m, dp_y5, nullptr);
    dp_stage(7, dp_y5, m, nullptr, nullptr);
    launch_dp_control(dI, n, dp_e, dp_hst, dp_acc, dp_cnt, dp_sched, dp_maxK, (double)N * dt, dp_ovf, st);
    ++nlaunch;
    dp_start();
  }

  llg_status forward_dp(const T* phi, const void* m0_v, double* J, void* mT) {
    cudaEventRecord(ev0, st);
    material(phi);
    cudaMemcpyAsync(m, m0_v, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(dp_ck, m0_v, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(jterm, 0, sizeof(double) * rt.size(), st);
    cudaMemsetAsync(slots, 0, sizeof(double) * total_slots, st);
    cudaMemsetAsync(dp_acc, 0, sizeof(int) * n, st);
    cudaMemsetAsync(dp_cnt, 0, sizeof(int) * n, st);
    cudaMemsetAsync(dp_ovf, 0, sizeof(int), st);
    const double Tend = (double)N * dt;
    {
      std::vector<double> h0(4 * (size_t)n);
      for (int i = 0; i < n; ++i) {
        const bool last = dt >= Tend;
        h0[4 * i] = 0.0;
        h0[4 * i + 1] = N > 0 ? (last ? Tend : dt) : 0.0;
        h0[4 * i + 2] = last ? 1.0 : 0.0;
        h0[4 * i + 3] = N > 0 ? 0.0 : 1.0;
      }
      cudaError_t e = cudaMemcpyAsync(dp_hst, h0.data(), sizeof(double) * h0.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "adaptive integrator: initial state");
    }
    // first attempt: k_1 = f(m, 0) and Y_2
    fft_only(m);
    dp_stage(1, m, m, Ya, nullptr);
    const long long max_att = 4 * std::max(1LL, N);
    std::vector<double> hh(4 * (size_t)n);
    int ovf = 0;
    bool done = N == 0;
    for (long long att = 0; !done && att < max_att; att += 4) {
      if (llg_status st2 = run_segment(SEG_DP_ATTEMPT, 4)) return st2;
      cudaMemcpyAsync(hh.data(), dp_hst, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(&ovf, dp_ovf, sizeof(int), cudaMemcpyDeviceToHost, st);
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "adaptive integrator");
      done = true;
      for (int i = 0; i < n; ++i) done &= hh[4 * i + 3] != 0.0;
      if (ovf) return fail(LLG_ETIMEOUT, "adaptive integrator: more accepted steps than checkpoint slots");
    }
    if (!done) return fail(LLG_ETIMEOUT, "adaptive integrator: no end of the interval within 4 nsteps attempts");
    dp_cnt_h.assign(n, 0);
    cudaMemcpyAsync(dp_cnt_h.data(), dp_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    // terminal: field of m_T, energies, lambda_T, explicit dJ/dpsi
    fft_only(m);
    cols();
    {
      RowArgs<T> a = row_args();
      a.Yin = m;
      a.lam = lam;
      a.psib = psib;
      a.psic = psic;
      a.jterm = jterm;
      a.psitile = psitile;
      a.psimom = psimom;
      a.wtab = wtab;
      rows(a, ROW_TERMINAL);
    }
    launch_reduce_slots(dI, n, slots, N + 1, jterm, psitile, psimom, Jd, st);
    ++nlaunch;
    mN_ptr = m;
    if (mT) cudaMemcpyAsync(mT, m, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
    cudaEventRecord(ev1, st);
    cudaMemcpyAsync(J, Jd, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    int herr = 0;
    cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "llg_forward");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "llg_forward");
    time_drain();
    if (herr) return fail(LLG_ETIMEOUT, "a bounded device wait ran out in llg_forward");
    float f = 0.f;
    cudaEventElapsedTime(&f, ev0, ev1);
    ms = f;
    have_fwd = true;
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(J[i])) return fail(LLG_ENONFINITE, "J is not finite for instance " + std::to_string(i));
    return LLG_OK;
  }

  // one reverse step of the Dormand-Prince sweep (reverse index in *step_base)
  void dp_reverse_step() {
    const long long S = (long long)slot();
    auto Yrec = [&](int s) { return dp_recY + (long long)(s - 1) * S; };   // Y_s, s = 2..6 (Y_1 = mrev)
    auto Brec = [&](int s) { return dp_recB + (long long)(s - 1) * S; };
    auto Ys = [&](int s) -> T* { return s == 1 ? dp_mrev : Yrec(s); };
    launch_dp_reverse_state(n, dp_sched, dp_cnt, step_base, dp_hst, dp_slot, dp_K > 1 ? dp_k0 : nullptr, st);
    launch_dp_gather<T>(dI, dRT, (int)rt.size(), dp_K > 1 ? dp_seg : dp_ck, S, dp_slot, dp_mrev, st);
    nlaunch += 2;
    fft_only(dp_mrev);
    for (int s = 1; s <= 6; ++s) {
      cols();
      RowArgs<T> a = dp_args(s);
      a.Yin = Ys(s);
      a.m = dp_mrev;
      a.Yout = s < 6 ? Yrec(s + 1) : dp_y5;
      a.Bout = Brec(s);
      rows(a, ROW_DP_STAGE);
    }
    int cur = 0;
    {
      AdjArgs<T> a = adj_args();
      a.hst = dp_hst;
      a.ebuf = dp_eta;
      a.kstride = S;
      a.stage = 6;
      a.seed_only = 1;
      a.dpb = (T)dp::b(6);
      a.Yprev = Ys(6);
      a.Bprev = Brec(6);
      a.BbarOut = bb[cur];
      adj_dp(a);
    }
    for (int s = 6; s >= 1; --s) {
      cols();
      AdjArgs<T> a = adj_args();
      a.hst = dp_hst;
      a.ebuf = dp_eta;
      a.kstride = S;
      a.stage = s;
      a.Ys = Ys(s);
      a.Bbar = bb[cur];
      a.BbarOut = bb[1 - cur];
      if (s > 1) {
        a.Yprev = Ys(s - 1);
        a.Bprev = Brec(s - 1);
        a.dpb = (T)dp::b(s - 1);
        for (int i = s; i <= 6; ++i) a.dpa[i] = (T)dp::a(i, s - 1);
      }
      adj_dp(a);
      if (s > 1) cur ^= 1;
    }
  }

  // replay step *step_base of a reverse block: every instance advances the
  // state in dp_mrev by its recorded step (or idles with h = 0) through the
  // six stages; the new state goes to dp_mrev and to segment slot j + 1
  void dp_replay_step() {
    const long long S = (long long)slot();
    auto Yrec = [&](int s) { return dp_recY + (long long)(s - 1) * S; };
    launch_dp_replay_state(n, dp_sched, step_base, dp_k0, dp_khi, dp_hst, st);
    ++nlaunch;
    fft_only(dp_mrev);
    for (int s = 1; s <= 6; ++s) {
      cols();
      RowArgs<T> a = dp_args(s);
      a.Yin = s == 1 ? dp_mrev : Yrec(s);
      a.m = dp_mrev;
      a.Yout = s < 6 ? Yrec(s + 1) : dp_y5;
      rows(a, ROW_DP_STAGE);
    }
    launch_dp_push<T>(dI, dRT, (int)rt.size(), dp_y5, dp_seg, S, step_base, dp_mrev, st);
    ++nlaunch;
  }

  // reverse sweep over the accepted steps: per reverse index r, instance i
  // reverses its step cnt_i - 1 - r (or idles with h = 0): recompute the six
  // stages from its state, seed kappa_6 = h b_6 lambda, then adjoint stages
  // 6..1 (eta_s kept for the lower stages, lambda += sum eta at 1).  With
  // periodic checkpoints the reverse indices go in blocks of dp_K: each block
  // first replays, per instance, the steps from the checkpoint at or before
  // its window to the window's end (at most 2 dp_K - 1 steps).
  llg_status adjoint_dp(const double* dw, void* dphi, void* dm0) {
    cudaEventRecord(ev0, st);
    long long Kmax = 0;
    for (int i = 0; i < n; ++i) Kmax = std::max(Kmax, (long long)dp_cnt_h[i]);
    for (long long b = 0; b * dp_K < Kmax; ++b) {
      if (dp_K > 1) {
        long long len = 0;   // replay steps this block needs (host copy of the plan)
        for (int i = 0; i < n; ++i) {
          const long long hi = (long long)dp_cnt_h[i] - 1 - b * dp_K;
          if (hi < 0) continue;
          const long long lo = std::max(0LL, (long long)dp_cnt_h[i] - (b + 1) * dp_K);
          len = std::max(len, hi - (lo / dp_K) * dp_K);
        }
        launch_dp_replay_plan(n, dp_cnt, b, dp_K, dp_k0, dp_khi, dp_ckslot, st);
        launch_dp_gather<T>(dI, dRT, (int)rt.size(), dp_ck, (long long)slot(), dp_ckslot, dp_mrev, st);
        set_step(-1);
        launch_dp_push<T>(dI, dRT, (int)rt.size(), dp_mrev, dp_seg, (long long)slot(), step_base, dp_mrev, st);
        nlaunch += 3;
        for (long long j = 0; j < len; ++j) {
          set_step(j);
          if (llg_status st2 = run_segment(SEG_DP_REPLAY, 1)) return st2;
        }
      }
      for (long long r = b * dp_K; r < std::min(Kmax, (b + 1) * dp_K); ++r) {
        set_step(r);
        if (llg_status st2 = run_segment(SEG_DP_REVERSE, 1)) return st2;
      }
    }
    launch_grad_finish_tiles<T>(dI, dRT, (int)rt.size(), dpsi, psib, psic, dw, static_cast<T*>(dphi), lam,
                                static_cast<T*>(dm0), st);
    ++nlaunch;
    cudaEventRecord(ev1, st);
    int herr = 0;
    cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "llg_adjoint");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "llg_adjoint");
    time_drain();
    if (herr) return fail(LLG_ETIMEOUT, "a bounded device wait ran out in llg_adjoint");
    float f = 0.f;
    cudaEventElapsedTime(&f, ev0, ev1);
    ms = f;
    have_fwd = false;
    return LLG_OK;
  }

  llg_status adaptive_steps(int inst, double* t, double* h, long long cap, long long* count) override {
    if (!dp_mode || dp_cnt_h.empty()) return fail(LLG_ESTATE, "no adaptive forward pass to report");
    if (inst < 0 || inst >= n || !count || cap < 0 || (cap > 0 && (!t || !h)))
      return fail(LLG_EINVAL, "adaptive_steps: bad instance or buffers");
    const long long K = dp_cnt_h[inst];
    *count = K;
    const long long k_n = std::min(K, cap);
    if (k_n == 0) return LLG_OK;
    std::vector<double> buf(2 * (size_t)n * k_n);
    cudaError_t e = cudaMemcpyAsync(buf.data(), dp_sched, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "adaptive_steps");
    for (long long k = 0; k < k_n; ++k) {
      t[k] = buf[2 * (k * n + inst)];
      h[k] = buf[2 * (k * n + inst) + 1];
    }
    return LLG_OK;
  }

  llg_status forward(const void* phi_v, const void* m0_v, double* J, void* mT) override {
    if (!phi_v || !m0_v || !J) return fail(LLG_EINVAL, "phi, m0 and J must not be NULL");
    if (dp_mode) return forward_dp(static_cast<const T*>(phi_v), m0_v, J, mT);
    const T* phi = static_cast<const T*>(phi_v);
    cudaEventRecord(ev0, st);
    material(phi);
    cudaMemcpyAsync(m, m0_v, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(slots, 0, sizeof(double) * total_slots, st);
    cudaMemsetAsync(jterm, 0, sizeof(double) * rt.size(), st);
    if (any_spec) cudaMemsetAsync(pslots, 0, sizeof(double) * 2 * total_slots, st);
    fft_only(m);
    const T* cur = m;
    for (const Action& ac : fwd) {
      if (ac.op == SNAP) {
        cudaMemcpyAsync(ckpt + (size_t)ac.b * slot(), m, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
      } else if (ac.op == ADVANCE) {
        set_step(ac.a);
        if (llg_status s = run_segment(SEG_ADVANCE, ac.b - ac.a)) return s;
        cur = m;
      } else if (ac.op == RECORD) {
        cudaMemcpyAsync(recY_slot(0), m, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
        set_step(ac.a);
        if (llg_status s = run_segment(SEG_RECORD_FWD, ac.b - ac.a)) return s;
        cur = Mrec(ac.b - ac.a);
      }
    }
    mN_ptr = cur;
    if (any_spec)
      if (llg_status s = spectral_weights()) return s;
    // terminal: field of m_N, energies, lambda_N, explicit dJ/dpsi
    cols();
    {
      RowArgs<T> a = row_args();
      a.Yin = cur;
      a.lam = lam;
      a.psib = psib;
      a.psic = psic;
      a.jterm = jterm;
      a.psitile = psitile;
      a.psimom = psimom;
      a.wtab = wtab;
      rows(a, ROW_TERMINAL);
    }
    launch_reduce_slots(dI, n, slots, N + 1, jterm, psitile, psimom, Jd, st);
    ++nlaunch;
    if (mT) cudaMemcpyAsync(mT, cur, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
    cudaEventRecord(ev1, st);
    cudaMemcpyAsync(J, Jd, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    int herr = 0;
    cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "llg_forward");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "llg_forward");
    time_drain();
    if (herr) return fail(LLG_ETIMEOUT, "a bounded device wait ran out in llg_forward");
    float f = 0.f;
    cudaEventElapsedTime(&f, ev0, ev1);
    ms = f;
    have_fwd = true;
    if (any_spec)
      for (int i = 0; i < n; ++i) J[i] += Jspec[i];
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(J[i])) return fail(LLG_ENONFINITE, "J is not finite for instance " + std::to_string(i));
    return LLG_OK;
  }

  // ------------------------------------------------------------ adjoint
  template <typename S = T>
  AdjArgs<T, S> adj_args() {
    AdjArgs<T, S> a;
    std::memset(&a, 0, sizeof a);
    a.inst = dI;
    a.tiles = dRT;
    if constexpr (std::is_same<S, T>::value) {
      a.spec = spec;
      a.tw = tw;
    } else {
      a.spec = spec_df;
      a.tw = tw_df;
    }
    a.psi = psi;
    a.gpart = gpart;
    a.lam = lam;
    a.G = G;
    a.psib = psib;
    a.psic = psic;
    a.step_base = step_base;
    a.err = errw;
    a.rows_max = R;
    a.dt = dt;
    a.n_from = n_from;
    a.wtab = wtab;
    return a;
  }
  void adj_dp(const AdjArgs<T>& a0) {
    AdjArgs<T> a = a0;
    time_begin(2);
    if (!rt2.empty()) {
      a.tiles = dRT2;
      launch_adj_dp<T>(a, (int)rt2.size(), smem_adj, st, false);
      ++nlaunch;
    }
    if (!rt3.empty()) {
      a.tiles = dRT3;
      launch_adj_dp<T>(a, (int)rt3.size(), smem_adj, st, true);
      ++nlaunch;
    }
    time_end(2);
  }
  // double-float row transforms of the split adjoint stage (dir +1: spec_df
  // -> Dbuf, dir -1: src -> spec_df)
  void spec_rows_df(int dir, const T* src) {
    if constexpr (std::is_same<T, float>::value) {
      SpecRowArgs<float, dfloat> r;
      r.inst = dI;
      r.spec = spec_df;
      r.tw = tw_df;
      r.out = Dbuf;
      r.src = src;
      r.err = errw;
      time_begin(4);
      const auto p2 = part(rt2.size(), split_rt2);
      if (p2.second) {
        r.tiles = (grp_sel < 0 ? dRT2 : dRT2p) + p2.first;
        launch_spec_rows<float, dfloat>(r, dir, (int)p2.second, smem_rows_df, st);
        ++nlaunch;
      }
      time_end(4);
    }
  }

  template <typename S>
  void adj(const AdjArgs<T, S>& a0) {
    if constexpr (!std::is_same<S, T>::value) {
      if (L.adj_split) {
        // inverse row transform of N * Bbar_s to Dbuf, the FP32 node phase,
        // then the forward row transform of the next Bbar
        AdjArgs<T> b = adj_args<T>();
        b.local_step = a0.local_step;
        b.stage = a0.stage;
        b.seed_only = a0.seed_only;
        b.seed_next = a0.seed_next;
        b.Ys = a0.Ys;
        b.Bbar = a0.Bbar;
        b.BbarOut = a0.BbarOut;
        b.Yprev = a0.Yprev;
        b.Bprev = a0.Bprev;
        b.Dext = Dbuf;
        if (!b.seed_only) spec_rows_df(1, nullptr);
        time_begin(2);
        const auto p2 = part(rt2.size(), split_rt2);
        if (p2.second) {
          b.tiles = (grp_sel < 0 ? dRT2 : dRT2p) + p2.first;
          launch_adj_split<T>(b, (int)p2.second, smem_split, st, L.adj_blocks);
          ++nlaunch;
        }
        time_end(2);
        if (b.seed_only || b.stage > 1 || b.seed_next) spec_rows_df(-1, b.BbarOut);
        return;
      }
    }
    AdjArgs<T, S> a = a0;
    const size_t sm = std::is_same<S, T>::value ? smem_adj : smem_adj_df;
    const int mb = std::is_same<S, T>::value ? 0 : L.adj_blocks;
    time_begin(2);
    const auto p2 = part(rt2.size(), split_rt2), p3 = part(rt3.size(), split_rt3);
    if (p2.second) {
      a.tiles = (grp_sel < 0 ? dRT2 : dRT2p) + p2.first;
      launch_adj<T, S>(a, (int)p2.second, sm, st, false, mb);
      ++nlaunch;
    }
    if (p3.second) {
      a.tiles = (grp_sel < 0 ? dRT3 : dRT3p) + p3.first;
      launch_adj<T, S>(a, (int)p3.second, sm, st, true, mb);
      ++nlaunch;
    }
    time_end(2);
  }

  // the per-instance cotangents (nullptr: all 1) for grad_finish
  llg_status upload_wext(const double* w, const double** dw) {
    *dw = nullptr;
    if (!w) return LLG_OK;
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(w[i])) return fail(LLG_EINVAL, "dJ_dextra must be finite");
    cudaError_t e = cudaMemcpyAsync(wext, w, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload dJ_dextra");
    *dw = wext;
    return LLG_OK;
  }

  llg_status adjoint(const double* w, void* dphi, void* dm0) override {
    if (!have_fwd) return fail(LLG_ESTATE, "llg_adjoint needs a preceding llg_forward");
    if (!dphi) return fail(LLG_EINVAL, "dJdphi must not be NULL");
    const double* dw = nullptr;
    if (llg_status s = upload_wext(w, &dw)) return s;
    if (dp_mode) return adjoint_dp(dw, dphi, dm0);
    cudaEventRecord(ev0, st);
    // The working state m (with the spectrum of its stage-1 input) is what
    // RESTORE loads, ADVANCE moves, SNAP saves and RECORD starts from.
    for (const Action& ac : rev) {
      if (ac.op == RESTORE) {
        cudaMemcpyAsync(m, ckpt + (size_t)ac.a * slot(), sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
        fft_only(m);
      } else if (ac.op == SNAP) {
        cudaMemcpyAsync(ckpt + (size_t)ac.b * slot(), m, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
      } else if (ac.op == ADVANCE) {
        set_step(ac.a);
        if (llg_status s = run_segment(SEG_ADVANCE_ADJ, ac.b - ac.a)) return s;
      } else if (ac.op == RECORD) {
        cudaMemcpyAsync(recY_slot(0), m, sizeof(T) * slot(), cudaMemcpyDeviceToDevice, st);
        set_step(ac.a);
        if (llg_status s = run_segment(SEG_RECORD_ADJ, ac.b - ac.a)) return s;
      } else if (ac.op == REVERSE) {
        set_step(ac.b);
        if (llg_status s = run_segment(SEG_REVERSE, ac.a - ac.b)) return s;
      }
    }
    launch_grad_finish_tiles<T>(dI, dRT, (int)rt.size(), dpsi, psib, psic, dw, static_cast<T*>(dphi), lam,
                                static_cast<T*>(dm0), st);
    ++nlaunch;
    cudaEventRecord(ev1, st);
    int herr = 0;
    cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "llg_adjoint");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "llg_adjoint");
    time_drain();
    if (herr) return fail(LLG_ETIMEOUT, "a bounded device wait ran out in llg_adjoint");
    float f = 0.f;
    cudaEventElapsedTime(&f, ev0, ev1);
    ms = f;
    have_fwd = false;
    return LLG_OK;
  }

  llg_status levelset(void* phi, const void* grad, const unsigned char* mask, double lr) override {
    if (!phi || !grad || !mask) return fail(LLG_EINVAL, "phi, grad and mask must not be NULL");
    cudaMemsetAsync(maxbits, 0, sizeof(unsigned int) * 2 * n, st);
    launch_levelset_tiles<T>(dI, dRT, (int)rt.size(), static_cast<T*>(phi), static_cast<const T*>(grad), mask,
                             lr, maxbits, st);
    nlaunch += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "levelset_step");
    return LLG_OK;
  }

  llg_status field(const void* phi, const void* mv, double t, int demag_only, void* B) override {
    if (!phi || !mv || !B) return fail(LLG_EINVAL, "phi, m and B must not be NULL");
    if (((uintptr_t)mv | (uintptr_t)B) % 16 != 0) return fail(LLG_EINVAL, "m and B must be 16-byte aligned");
    have_fwd = false;
    material(static_cast<const T*>(phi));
    fft_only(static_cast<const T*>(mv));
    cols();
    RowArgs<T> a = row_args();
    a.Yin = static_cast<const T*>(mv);
    a.Bout = static_cast<T*>(B);
    a.t_field = t;
    a.demag_only = demag_only;
    rows(a, ROW_FIELD);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "llg_field");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "llg_field");
    return LLG_OK;
  }
};

// ---------------------------------------------------------------- C ABI

extern "C" {

llg_status llg_create(const llg_problem* inst, int n_inst, const llg_options* opt, void* cuda_stream,
                      llg_ctx** out) {
  if (!out) return LLG_EINVAL;
  *out = nullptr;
  if (!inst || n_inst <= 0) return LLG_EINVAL;
  llg_options o;
  if (opt) {
    o = *opt;
  } else {
    std::memset(&o, 0, sizeof o);
    o.precision = LLG_FP32;
    o.ckpt = LLG_CKPT_PERIODIC;
  }
  llg_ctx* ctx = nullptr;
  llg_status s;
  if (o.precision == LLG_FP64) {
    auto* e = new Engine<double>();
    s = e->create(inst, n_inst, &o, static_cast<cudaStream_t>(cuda_stream));
    ctx = e;
  } else {
    auto* e = new Engine<float>();
    s = e->create(inst, n_inst, &o, static_cast<cudaStream_t>(cuda_stream));
    ctx = e;
  }
  *out = ctx;   // returned even on failure so that llg_last_error can explain it
  return s;
}

llg_status llg_forward(llg_ctx* ctx, const void* phi_dev, const void* m0_dev, double* J_host, void* mT_dev) {
  if (!ctx) return LLG_EINVAL;
  return ctx->forward(phi_dev, m0_dev, J_host, mT_dev);
}

llg_status llg_adjoint(llg_ctx* ctx, const double* dJ_dextra, void* dJdphi_dev, void* dJdm0_dev) {
  if (!ctx) return LLG_EINVAL;
  return ctx->adjoint(dJ_dextra, dJdphi_dev, dJdm0_dev);
}

llg_status llg_launch_config(llg_ctx* ctx, llg_launch* out, double* tune_ms) {
  if (!ctx || !out) return LLG_EINVAL;
  *out = ctx->L;
  if (tune_ms) *tune_ms = ctx->tune_ms;
  return LLG_OK;
}

llg_status llg_adaptive_steps(llg_ctx* ctx, int inst, double* t_host, double* h_host, long long cap,
                              long long* count) {
  if (!ctx) return LLG_EINVAL;
  return ctx->adaptive_steps(inst, t_host, h_host, cap, count);
}

llg_status levelset_step(llg_ctx* ctx, void* phi_dev, const void* grad_dev, const unsigned char* mask_dev,
                         double lr) {
  if (!ctx) return LLG_EINVAL;
  return ctx->levelset(phi_dev, grad_dev, mask_dev, lr);
}

llg_status llg_field(llg_ctx* ctx, const void* phi_dev, const void* m_dev, double t, int demag_only,
                     void* B_dev) {
  if (!ctx) return LLG_EINVAL;
  return ctx->field(phi_dev, m_dev, t, demag_only, B_dev);
}

llg_status llg_query(llg_ctx* ctx, size_t* device_bytes, double* last_ms) {
  if (!ctx) return LLG_EINVAL;
  if (device_bytes) *device_bytes = ctx->device_bytes();
  if (last_ms) *last_ms = ctx->last_ms();
  return LLG_OK;
}

long long llg_launch_count(llg_ctx* ctx) { return ctx ? ctx->launches() : 0; }

llg_status llg_kernel_time(llg_ctx* ctx, int family, long long* launches, double* total_ms) {
  if (!ctx || family < 0 || family > 4) return LLG_EINVAL;
  ctx->kernel_time(family, launches, total_ms);
  return LLG_OK;
}

const char* llg_last_error(llg_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void llg_destroy(llg_ctx* ctx) { delete ctx; }

long long llg_schedule(long long nsteps, int ckpt, int seg_len, long long* actions, long long max_actions,
                       long long* n_forward) {
  if (nsteps < 0 || seg_len < 0 ||
      (ckpt != LLG_CKPT_PERIODIC && ckpt != LLG_CKPT_STORE_ALL && ckpt != LLG_CKPT_BINOMIAL))
    return -1;
  std::vector<Action> f, r;
  make_schedule(nsteps, ckpt, seg_len, f, r);
  const long long tot = (long long)(f.size() + r.size());
  if (n_forward) *n_forward = (long long)f.size();
  if (actions) {
    long long k = 0;
    for (const Action& a : f) {
      if (k >= max_actions) break;
      actions[3 * k] = a.op; actions[3 * k + 1] = a.a; actions[3 * k + 2] = a.b;
      ++k;
    }
    for (const Action& a : r) {
      if (k >= max_actions) break;
      actions[3 * k] = a.op; actions[3 * k + 1] = a.a; actions[3 * k + 2] = a.b;
      ++k;
    }
  }
  return tot;
}

int llg_padded_extents(int nx, int ny, int* Px, int* Py) {
  if (nx < 1 || ny < 1) return -1;
  if (Px) *Px = std::max(16, next_pow2(2 * nx));
  if (Py) *Py = std::max(8, next_pow2(2 * ny));
  return 0;
}

int llg_abi_version(void) { return 2; }

}  // extern "C"
