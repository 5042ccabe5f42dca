// C ABI of libddelm (declared in include/ddelm.h): handle creation, the setup
// sequence (assembly, shifted CholeskyQR3 of every local least-squares
// matrix, local operators, coarse problem), the solve sequence and
// inspection.  The library allocates no device memory: every buffer lives in
// the caller's workspace.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "ddelm_internal.h"

using namespace ddelm;

namespace ddelm {
std::atomic<long long> g_kernel_launches{0};
namespace {
thread_local char g_last_error[512] = "";
}
void record_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  const char *f = std::strrchr(file, '/');
  std::snprintf(g_last_error, sizeof(g_last_error), "%s (%s) in %s at %s:%d", cudaGetErrorName(e),
                cudaGetErrorString(e), what, f ? f + 1 : file, line);
}
void record_plan_error(const std::string &why) {
  std::snprintf(g_last_error, sizeof(g_last_error), "problem rejected: %s", why.empty() ? "invalid plan" : why.c_str());
}
}  // namespace ddelm

struct ddelm_handle {
  Plan plan;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  // CUDA graphs of the setup and of the solve sequence (captured on second use)
  cudaGraphExec_t setup_exec = nullptr, solve_exec = nullptr;
  long long solves = 0;
  bool fwd_valid = false;  // the solve staging holds the data and solution of the last ddelm_solve
  bool graph_off = false;  // capture unavailable (or disabled by the options)
  // tile-shape autotuner: pending until the first setup has run; its outcome
  bool tune_pending = false, capturing = false;
  int tune_phases = 0, tune_switched = 0;
  double tune_ms_rule = 0.0, tune_ms_chosen = 0.0;
  std::vector<double> tune_log;  // per timed phase: index, rule width, its ms, alternative width, its ms
  // profiling: event pairs around launches, reduced on ddelm_profile
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_cls;
  size_t ev_used = 0;
  double prof_ms[DDELM_PROF_CLASSES] = {};
  long long prof_n[DDELM_PROF_CLASSES] = {};
  std::vector<long long> ev_kernels;  // kernels launched inside each recorded pair
};

namespace {

#define CK(x)                                                 \
  do {                                                        \
    cudaError_t e_ = (x);                                     \
    if (e_ != cudaSuccess) {                                  \
      ::ddelm::record_cuda_error(e_, #x, __FILE__, __LINE__); \
      return DDELM_ERR_CUDA;                                  \
    }                                                         \
  } while (0)

double *dbase(ddelm_handle *h) { return reinterpret_cast<double *>(h->ws + h->plan.off_dbl); }

// Records an event pair around a launch when profiling is on.
struct ProfScope {
  ddelm_handle *h;
  cudaStream_t s;
  size_t k = (size_t)-1;
  long long n0 = 0;
  ProfScope(ddelm_handle *h_, int cls, cudaStream_t s_) : h(h_), s(s_) {
    if (!h->prof) return;
    if (h->ev_used + 2 > h->ev.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
      h->ev.push_back(a);
      h->ev.push_back(b);
      h->ev_cls.push_back(cls);
      h->ev_cls.push_back(cls);
      h->ev_kernels.push_back(0);
      h->ev_kernels.push_back(0);
    }
    k = h->ev_used;
    h->ev_used += 2;
    h->ev_cls[k] = cls;
    n0 = ddelm::g_kernel_launches.load(std::memory_order_relaxed);
    cudaEventRecord(h->ev[k], s);
  }
  ~ProfScope() {
    if (k == (size_t)-1) return;
    cudaEventRecord(h->ev[k + 1], s);
    h->ev_kernels[k] = ddelm::g_kernel_launches.load(std::memory_order_relaxed) - n0;
  }
};

enum { PC_FEAT = 0, PC_GEMM = 1, PC_CHOL = 2, PC_CG = 3, PC_OTHER = 4, PC_SLICE = 5, PC_TC = 6 };

#define LAUNCH(cls, call)              \
  do {                                 \
    ProfScope ps_(h, cls, s);          \
    CK(call);                          \
  } while (0)

template <class T>
void put(char *buf, size_t off, const std::vector<T> &v) {
  if (!v.empty()) std::memcpy(buf + off, v.data(), v.size() * sizeof(T));
}

// 2^(-j/256), j < 256, for the feature tanh (computed once per process)
const std::vector<double> &exp2_table() {
  static const std::vector<double> t = [] {
    std::vector<double> v(256);
    for (int j = 0; j < 256; ++j) v[j] = double(std::exp2l(-(long double)j / 256.0L));
    return v;
  }();
  return t;
}

// Host staging of an upload: one page-locked buffer per process, grown on
// demand and reused by every setup (a setup waits for its copies before it
// lets the buffer go); pageable memory when page-locked memory is refused.
struct Staging {
  std::mutex m;
  char *pinned = nullptr;
  size_t cap = 0;
};
Staging &staging() {
  static Staging st;
  return st;
}

int upload(ddelm_handle *h, const ddelm_problem *prob, cudaStream_t s) {
  Plan &p = h->plan;
  const long long sumM = p.sz.sum_M, sumI = p.sz.sum_int;
  const bool diff = p.op == DDELM_OP_DIFFUSION;
  // staging layout: the tables, then w, b, the feature constants, the exp2
  // table, the interior points (and the coefficient and its gradient)
  const size_t n_w = 2 * sumM, n_b = sumM, n_fc = 4 * sumM, n_x = sumI > 0 ? 2 * sumI : 0;
  const size_t n_a = (sumI > 0 && diff) ? sumI : 0, n_ga = (sumI > 0 && diff) ? 2 * sumI : 0;
  const size_t o_w = (p.bytes_tables + 15) / 16 * 16, o_b = o_w + 8 * n_w, o_fc = o_b + 8 * n_b,
               o_ex = o_fc + 8 * n_fc, o_x = o_ex + 8 * 256, o_a = o_x + 8 * n_x, o_ga = o_a + 8 * n_a,
               total = o_ga + 8 * n_ga;
  Staging &st = staging();
  std::lock_guard<std::mutex> lock(st.m);
  std::vector<char> pageable;
  // Whatever the return path, the stream is drained before the lock is released
  // (the guard is destroyed first): a copy that fails after others were queued
  // must not let the next setup refill the buffer while they still read it.
  struct DrainOnExit {
    cudaStream_t s;
    ~DrainOnExit() { (void)cudaStreamSynchronize(s); }
  } drain{s};
  char *buf = nullptr;
  if (st.cap < total) {
    if (st.pinned) cudaFreeHost(st.pinned);
    st.pinned = nullptr;
    st.cap = 0;
    const size_t want = total + total / 4;
    if (cudaHostAlloc(reinterpret_cast<void **>(&st.pinned), want, cudaHostAllocDefault) == cudaSuccess)
      st.cap = want;
    else {
      st.pinned = nullptr;
      (void)cudaGetLastError();
    }
  }
  if (st.pinned) {
    buf = st.pinned;
  } else {
    pageable.resize(total);
    buf = pageable.data();
  }
  put(buf, p.off_subs, p.subs);
  put(buf, p.off_rows, p.rows);
  put(buf, p.off_gdesc, p.gdesc);
  put(buf, p.off_gtile, p.gtile);
  put(buf, p.off_cdesc, p.cdesc);
  put(buf, p.off_mdesc, p.mdesc);
  put(buf, p.off_conv, p.conv);
  put(buf, p.off_ints, p.ints);
  put(buf, p.off_sdesc, p.sdesc);
  put(buf, p.off_odesc, p.odesc);
  put(buf, p.off_otile, p.otile);
  put(buf, p.off_ssubs, p.ssubs);
  put(buf, p.off_srows, p.srows);
  put(buf, p.off_scsub, p.scsub);
  put(buf, p.off_dots, p.dots);
  if (p.mixed) {
    std::vector<unsigned char> maps;
    const int rc = encode_tensor_maps(p, h->ws, maps);
    if (rc != DDELM_OK) return rc;
    std::memcpy(buf + p.off_tmaps, maps.data(), maps.size());
  }
  // problem data: w = s*w_hat, b = s*b_hat; the kernels evaluate tanh(u / 2)
  // at u = 2 (w . x + b), with the per-neuron constants (2 w, 2 b, 2 |w|^2)
  double *w = reinterpret_cast<double *>(buf + o_w), *b = reinterpret_cast<double *>(buf + o_b);
  double *fc = reinterpret_cast<double *>(buf + o_fc);
  for (long long j = 0; j < 2 * sumM; ++j) w[j] = prob->scale * prob->w_hat[j];
  for (long long j = 0; j < sumM; ++j) b[j] = prob->scale * prob->b_hat[j];
  for (long long j = 0; j < sumM; ++j) {
    fc[4 * j] = 2.0 * w[2 * j];
    fc[4 * j + 1] = 2.0 * w[2 * j + 1];
    fc[4 * j + 2] = 2.0 * b[j];
    fc[4 * j + 3] = 2.0 * (w[2 * j] * w[2 * j] + w[2 * j + 1] * w[2 * j + 1]);
  }
  std::memcpy(buf + o_ex, exp2_table().data(), 8 * 256);
  if (n_x) std::memcpy(buf + o_x, prob->x_int, 8 * n_x);
  if (n_a) std::memcpy(buf + o_a, prob->a_int, 8 * n_a);
  if (n_ga) std::memcpy(buf + o_ga, prob->grad_a_int, 8 * n_ga);
  double *db = dbase(h);
  CK(cudaMemcpyAsync(h->ws, buf, p.bytes_tables, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(db + p.o_w, buf + o_w, 8 * n_w, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(db + p.o_b, buf + o_b, 8 * n_b, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(db + p.o_fc, buf + o_fc, 8 * n_fc, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(db + p.o_exp2, buf + o_ex, 8 * 256, cudaMemcpyHostToDevice, s));
  if (n_x) CK(cudaMemcpyAsync(db + p.o_xint, buf + o_x, 8 * n_x, cudaMemcpyHostToDevice, s));
  if (n_a) CK(cudaMemcpyAsync(db + p.o_aint, buf + o_a, 8 * n_a, cudaMemcpyHostToDevice, s));
  if (n_ga) CK(cudaMemcpyAsync(db + p.o_gaint, buf + o_ga, 8 * n_ga, cudaMemcpyHostToDevice, s));
  // the staging buffer is released (and may be refilled) only after the copies
  CK(cudaStreamSynchronize(s));
  return DDELM_OK;
}

// Assembly, shifted CholeskyQR of [K; eps I] and [K-bar; eps-bar I] (the
// plan's step list, wave by wave), local operators and the coarse problem, all
// from workspace-resident data.
// Runs enqueue() on s, through a CUDA graph captured on first use (*exec), so
// that a repeated sequence of launches costs one graph launch.  Profiling
// (events around launches), the legacy default stream, or a failed capture run
// the sequence directly.
template <class F>
int run_graph(ddelm_handle *h, cudaStream_t s, cudaGraphExec_t *exec, F enqueue) {
  if (!s || h->prof || h->graph_off) return enqueue();
  if (!*exec) {
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      h->graph_off = true;
      return enqueue();
    }
    const int rc = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    cudaGraphExec_t x = nullptr;
    const bool ok = rc == DDELM_OK && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      (void)cudaGetLastError();
      h->graph_off = true;
      return enqueue();
    }
    *exec = x;
  }
  CK(cudaGraphLaunch(*exec, s));
  return DDELM_OK;
}

int enqueue_setup(ddelm_handle *h, cudaStream_t s);

// capture: false for a one-off setup (capturing would only add its cost)
int compute_setup(ddelm_handle *h, cudaStream_t s, int *info_sub, bool capture) {
  Plan &p = h->plan;
  double *db = dbase(h);
  {
    h->capturing = capture;
    const int rc = capture ? run_graph(h, s, &h->setup_exec, [&] { return enqueue_setup(h, s); })
                           : enqueue_setup(h, s);
    h->capturing = false;
    if (rc != DDELM_OK) return rc;
    if (!capture) h->tune_pending = false;  // the first direct setup has tuned every phase it could
  }
  CK(cudaStreamSynchronize(s));
  int oz_err = 0;
  CK(cudaMemcpy(&oz_err, db + p.o_status + 2 * p.n_sub + 32, sizeof(int), cudaMemcpyDeviceToHost));
  if (oz_err) return DDELM_ERR_TIMEOUT;
  std::vector<int> st(2 * (size_t)p.n_sub + 1);
  CK(cudaMemcpy(st.data(), db + p.o_status, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < st.size(); ++k)
    if (st[k]) {
      if (info_sub) *info_sub = int(k / 2);
      return DDELM_ERR_RANK_DEFICIENT;
    }
  return DDELM_OK;
}

// Choices of the tile-shape autotuner, kept for the life of the process and
// shared by every handle: the key is the phase's shape (its products' sizes,
// levels and triangular flags, and the tile options), so a later handle with
// the same phases (a new setup of the same problem) plans the chosen tile list
// alone instead of timing again.
std::mutex g_tune_mutex;
std::unordered_map<unsigned long long, int> g_tune_bn;

}  // namespace

int ddelm::tuned_tile_width(unsigned long long key) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune_bn.find(key);
  return it == g_tune_bn.end() ? 0 : it->second;
}

namespace {

// Every launch and copy of the setup, in stream order (no host synchronisation).
int enqueue_setup(ddelm_handle *h, cudaStream_t s) {
  Plan &p = h->plan;
  double *db = dbase(h);
  CK(cudaMemsetAsync(db + p.o_status, 0, (4 * (size_t)p.n_sub + 64) * 8, s));
  const long long np = p.n_pi > 0 ? p.n_pi : 1;
  CK(cudaMemsetAsync(db + p.o_Dpp, 0, np * np * 8, s));
  CK(cudaMemsetAsync(db + p.o_Spi, 0, np * np * 8, s));
  const auto &G = p.setup_gemm;
  // a setup GEMM phase runs on the tensor cores (BF16 slices) in MIXED precision
  auto gemm = [&](int q) -> int {
    if (p.mixed && q < (int)p.oz_phase.size() && p.oz_phase[q].ntile > 0) {
      OzPhase &ph = p.oz_phase[q];
      LAUNCH(PC_SLICE, launch_slices(p, ph, h->ws, s));
      if (h->tune_pending && !h->capturing && ph.overwrite && ph.ntile_alt > 0) {
        // autotuner: the other tile width, then the rule's (whose output stays);
        // the faster is kept for every later setup (and the captured graph)
        const unsigned long long key = ph.key;
        const int known = tuned_tile_width(key);
        if (known) {  // timed before in this process: apply the choice
          if (known != ph.bn) {
            std::swap(ph.tile0, ph.tile0_alt);
            std::swap(ph.ntile, ph.ntile_alt);
            std::swap(ph.bn, ph.bn_alt);
            std::swap(ph.flops, ph.flops_alt);
            p.oz_flops += ph.flops - ph.flops_alt;
            h->tune_switched++;
          }
          h->tune_phases++;
          LAUNCH(PC_TC, launch_oz_gemm(p, ph, h->ws, s));
          return DDELM_OK;
        }
        CK(preload_oz_kernels());  // no lazy module load inside the timed launches
        OzPhase alt = ph;
        alt.tile0 = ph.tile0_alt;
        alt.ntile = ph.ntile_alt;
        alt.bn = ph.bn_alt;
        cudaEvent_t ev[4] = {};
        for (auto &e : ev) CK(cudaEventCreate(&e));
        CK(cudaEventRecord(ev[0], s));
        LAUNCH(PC_TC, launch_oz_gemm(p, alt, h->ws, s));
        CK(cudaEventRecord(ev[1], s));
        CK(cudaEventRecord(ev[2], s));
        LAUNCH(PC_TC, launch_oz_gemm(p, ph, h->ws, s));
        CK(cudaEventRecord(ev[3], s));
        CK(cudaEventSynchronize(ev[3]));
        float t_alt = 0.f, t_rule = 0.f;
        CK(cudaEventElapsedTime(&t_alt, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&t_rule, ev[2], ev[3]));
        for (auto &e : ev) CK(cudaEventDestroy(e));
        h->tune_phases++;
        h->tune_ms_rule += t_rule;
        for (double v : {(double)q, (double)ph.bn, (double)t_rule, (double)alt.bn, (double)t_alt}) h->tune_log.push_back(v);
        const bool take_alt = t_alt < 0.97f * t_rule;  // a clear gain only: one run's timings carry noise
        {
          std::lock_guard<std::mutex> lk(g_tune_mutex);
          g_tune_bn[key] = take_alt ? alt.bn : ph.bn;
        }
        if (take_alt) {
          std::swap(ph.tile0, ph.tile0_alt);
          std::swap(ph.ntile, ph.ntile_alt);
          std::swap(ph.bn, ph.bn_alt);
          std::swap(ph.flops, ph.flops_alt);
          p.oz_flops += ph.flops - ph.flops_alt;
          h->tune_switched++;
          h->tune_ms_chosen += t_alt;
          LAUNCH(PC_TC, launch_oz_gemm(p, ph, h->ws, s));  // the kept width's output
        } else {
          h->tune_ms_chosen += t_rule;
        }
        return DDELM_OK;
      }
      LAUNCH(PC_TC, launch_oz_gemm(p, ph, h->ws, s));
    } else {
      LAUNCH(PC_GEMM, launch_gemm_phase(p, G[q], h->ws, s));
    }
    return DDELM_OK;
  };
  for (const Step &st : p.steps) {
    switch (st.kind) {
      case STEP_FEAT: {
        LAUNCH(PC_FEAT, launch_features(p, h->ws, st.idx, s));
        if (p.keep) {  // copies of the assembled matrices of this wave
          long long off = p.o_keepX;
          for (int i = 0; i < p.n_sub; ++i) {
            const SubDev &d = p.subs[i];
            const size_t mm = (size_t)d.m * d.M;
            if (i / p.wave == st.idx) {
              CK(cudaMemcpyAsync(db + off, db + d.oK, mm * 8, cudaMemcpyDeviceToDevice, s));
              CK(cudaMemcpyAsync(db + off + mm, db + d.oKb, mm * 8, cudaMemcpyDeviceToDevice, s));
              CK(cudaMemcpyAsync(db + off + 2 * mm, db + d.oA, (size_t)d.nG * d.M * 8, cudaMemcpyDeviceToDevice,
                                 s));
            }
            off += (2 * (long long)mm + (long long)d.nG * d.M + 31) / 32 * 32;
          }
        }
        break;
      }
      case STEP_GEMM: {
        const int rc = gemm(st.idx);
        if (rc != DDELM_OK) return rc;
        break;
      }
      case STEP_CHOL:
        LAUNCH(PC_CHOL, launch_chol_phase(p, p.chol_passes[st.idx], h->ws, s));
        break;
      case STEP_MATOP:
        LAUNCH(PC_OTHER, launch_matop_phase(p, p.matop_phases[st.idx], h->ws, s));
        break;
      default:
        return DDELM_ERR_INVALID_ARG;
    }
  }
  if (p.n_pi > 0) {
    LAUNCH(PC_OTHER, launch_coarse_assembly(p, h->ws, s));
    LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_coarse + 0], h->ws, s));
    CK(cudaMemcpyAsync(db + p.o_SpiR, db + p.o_Spi, (size_t)np * np * 8, cudaMemcpyDeviceToDevice, s));
    LAUNCH(PC_CHOL, launch_chol_phase(p, p.chol_coarse, h->ws, s));
    LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_coarse + 1], h->ws, s));
    LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_coarse + 2], h->ws, s));
    LAUNCH(PC_OTHER, launch_fill_identity(db + p.o_C2, p.n_pi, 1.0, s));
    LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_coarse + 3], h->ws, s));
  }
  if (p.mixed) LAUNCH(PC_OTHER, launch_convert_f32(p, h->ws, s));  // operators of the inner FP32 CG
  return DDELM_OK;
}

}  // namespace

extern "C" {

int ddelm_query(const ddelm_problem *prob, ddelm_sizes *out) {
  ddelm::g_last_error[0] = '\0';
  if (!out) return DDELM_ERR_INVALID_ARG;
  Plan p;
  int rc = build_plan(prob, p);
  if (rc != DDELM_OK) {
    record_plan_error(p.err);
    return rc;
  }
  *out = p.sz;
  return DDELM_OK;
}

int ddelm_setup(const ddelm_problem *prob, void *d_workspace, size_t workspace_bytes, void *stream,
                ddelm_handle **out, int *info_sub) {
  ddelm::g_last_error[0] = '\0';
  if (!out || !d_workspace) return DDELM_ERR_INVALID_ARG;
  *out = nullptr;
  if (info_sub) *info_sub = -1;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return DDELM_ERR_INVALID_ARG;
  ddelm_handle *h = new (std::nothrow) ddelm_handle();
  if (!h) return DDELM_ERR_INVALID_ARG;
  int rc = build_plan(prob, h->plan);
  if (rc != DDELM_OK) {
    record_plan_error(h->plan.err);
    delete h;
    return rc;
  }
  h->graph_off = prob->opt.disable_graphs != 0;
  h->tune_pending = prob->opt.autotune != 0 && prob->opt.precision == DDELM_PREC_MIXED;
  if (workspace_bytes < h->plan.bytes_total) {
    delete h;
    return DDELM_ERR_INVALID_ARG;
  }
  h->ws = static_cast<char *>(d_workspace);
  h->ws_bytes = workspace_bytes;
  rc = upload(h, prob, static_cast<cudaStream_t>(stream));
  if (rc == DDELM_OK) rc = compute_setup(h, static_cast<cudaStream_t>(stream), info_sub, false);
  if (rc == DDELM_ERR_RANK_DEFICIENT && h->plan.dw_auto) {
    // the automatic double-FP32 first factors were not accurate enough for this
    // problem: FP64 factors (the CQR2_SERIES scheme) and the setup again
    Plan &p = h->plan;
    for (const auto &fb : p.dw_fallback) {
      p.cdesc[fb.first].prec = 0;
      p.cdesc[fb.first].shift_rel = fb.second;
    }
    p.scheme = DDELM_SCHEME_CQR2_SERIES;
    p.dw_auto = false;
    const cudaError_t e = cudaMemcpy(h->ws + p.off_cdesc, p.cdesc.data(), p.cdesc.size() * sizeof(CholDesc),
                                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      record_cuda_error(e, "cudaMemcpy(cdesc)", __FILE__, __LINE__);
      rc = DDELM_ERR_CUDA;
    } else {
      if (info_sub) *info_sub = -1;
      rc = compute_setup(h, static_cast<cudaStream_t>(stream), info_sub, false);
    }
  }
  if (rc != DDELM_OK && rc != DDELM_ERR_RANK_DEFICIENT) {
    ddelm_destroy(h);
    return rc;
  }
  *out = h;
  return rc;
}

int ddelm_refactor(ddelm_handle *h, void *stream, int *info_sub) {
  if (!h) return DDELM_ERR_INVALID_ARG;
  if (info_sub) *info_sub = -1;
  h->fwd_valid = false;
  return compute_setup(h, static_cast<cudaStream_t>(stream), info_sub, true);
}

int ddelm_solve(ddelm_handle *h, const double *d_f_int, const double *d_g_bnd, double *d_c, double *d_mu,
                double *d_u_eval, ddelm_solve_info *info, void *stream) {
  if (!h) return DDELM_ERR_INVALID_ARG;
  Plan &p = h->plan;
  if ((p.sz.sum_int > 0 && !d_f_int) || (p.sz.n_bnd > 0 && !d_g_bnd)) return DDELM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *db = dbase(h);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (info) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
  }
  // the caller's data in, through the staging buffers (fixed addresses)
  const int R = p.n_rhs;
  if (p.sz.sum_int > 0) CK(cudaMemcpyAsync(db + p.o_fin, d_f_int, (size_t)p.sz.sum_int * R * 8, cudaMemcpyDeviceToDevice, s));
  if (p.sz.n_bnd > 0) CK(cudaMemcpyAsync(db + p.o_gin, d_g_bnd, (size_t)p.sz.n_bnd * R * 8, cudaMemcpyDeviceToDevice, s));
  auto enqueue = [&]() -> int {
    LAUNCH(PC_OTHER, launch_gather_rhs(p, h->ws, db + p.o_fin, db + p.o_gin, s));
    const auto &G = p.setup_gemm;
    for (int q = 0; q < 4; ++q) LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_solve + q], h->ws, s));
    // barrier words and error flag
    CK(cudaMemsetAsync(db + p.o_status + 2 * p.n_sub + 8, 0, 16 * 8, s));
    CgArgs a;
    a.mu_out = db + p.o_muout;
    a.c_out = db + p.o_cout;
    a.max_iters = p.opt.max_iters;
    a.tol = p.opt.tol;
    a.theta = p.opt.theta;
    a.max_refine = p.opt.max_refine;
    LAUNCH(PC_CG, launch_cg(p, h->ws, a, s));
    if (p.sz.sum_eval > 0) {
      LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_solve + 4], h->ws, s));
      for (const auto &d : p.subs)
        if (d.nE > 0)
          CK(cudaMemcpyAsync(db + p.o_uout + d.eval_off * R, db + d.oU, (size_t)d.nE * R * 8,
                             cudaMemcpyDeviceToDevice, s));
    }
    return DDELM_OK;
  };
  {
    // a handle's first solve runs directly; later ones replay one captured graph
    h->fwd_valid = false;
    const int rc0 = h->solves++ == 0 ? enqueue() : run_graph(h, s, &h->solve_exec, enqueue);
    if (rc0 != DDELM_OK) return rc0;
    h->fwd_valid = true;
  }
  // results out
  if (d_c) CK(cudaMemcpyAsync(d_c, db + p.o_cout, (size_t)p.sz.sum_M * R * 8, cudaMemcpyDeviceToDevice, s));
  if (d_mu)
    CK(cudaMemcpyAsync(d_mu, db + p.o_muout, (size_t)(p.n_pi + p.n_dl) * R * 8, cudaMemcpyDeviceToDevice, s));
  if (d_u_eval && p.sz.sum_eval > 0)
    CK(cudaMemcpyAsync(d_u_eval, db + p.o_uout, (size_t)p.sz.sum_eval * R * 8, cudaMemcpyDeviceToDevice, s));
  int rc = DDELM_OK;
  double hinfo[40];
  int herr = 0;
  if (info) CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  const long long nd = p.n_dl > 0 ? p.n_dl : 1, np = p.n_pi > 0 ? p.n_pi : 1;
  const double *info_dev = db + p.o_cg + 12 * nd * p.n_rhs + 14 * np * p.n_rhs + 2048 * 32 - 64;
  CK(cudaMemcpy(hinfo, info_dev, sizeof(hinfo), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&herr, db + p.o_status + 2 * p.n_sub + 16, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) rc = DDELM_ERR_TIMEOUT;
  const int iters = int(hinfo[0]);
  double resmax = 0.0;
  bool finite = true;
  for (int k = 0; k < p.n_rhs; ++k) {
    resmax = hinfo[1 + k] > resmax ? hinfo[1 + k] : resmax;
    finite = finite && std::isfinite(hinfo[1 + k]) && std::isfinite(hinfo[17 + k]);
  }
  if (rc == DDELM_OK && iters >= p.opt.max_iters && !(resmax < p.opt.tol)) rc = DDELM_ERR_NOT_CONVERGED;
  if (rc == DDELM_OK && !finite) rc = DDELM_ERR_NOT_CONVERGED;  // NaN or Inf in the data or the iteration
  if (!finite) resmax = std::numeric_limits<double>::quiet_NaN();
  if (info) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    info->iterations = iters;
    info->refinements = p.mixed ? int(hinfo[33]) : 0;
    info->rel_residual = resmax;
    info->ms_total = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return rc;
}

int ddelm_interface_residual(ddelm_handle *h, const double *d_f_int, const double *d_g_bnd,
                             const double *d_mu_delta, double *d_r, double *d_c, double *d_u_eval, void *stream) {
  if (!h || !d_mu_delta) return DDELM_ERR_INVALID_ARG;
  Plan &p = h->plan;
  if ((p.sz.sum_int > 0 && !d_f_int) || (p.sz.n_bnd > 0 && !d_g_bnd)) return DDELM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *db = dbase(h);
  const int R = p.n_rhs;
  double *mu = nullptr, *rhs = nullptr, *res = nullptr;
  cg_vectors(p, h->ws, &mu, &rhs, &res);
  h->fwd_valid = false;  // the staging now holds this call's data
  if (p.sz.sum_int > 0) CK(cudaMemcpyAsync(db + p.o_fin, d_f_int, (size_t)p.sz.sum_int * R * 8, cudaMemcpyDeviceToDevice, s));
  if (p.sz.n_bnd > 0) CK(cudaMemcpyAsync(db + p.o_gin, d_g_bnd, (size_t)p.sz.n_bnd * R * 8, cudaMemcpyDeviceToDevice, s));
  if (p.n_dl > 0) CK(cudaMemcpyAsync(mu, d_mu_delta, (size_t)p.n_dl * R * 8, cudaMemcpyDeviceToDevice, s));
  LAUNCH(PC_OTHER, launch_gather_rhs(p, h->ws, db + p.o_fin, db + p.o_gin, s));
  const auto &G = p.setup_gemm;
  for (int q = 0; q < 4; ++q) LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_solve + q], h->ws, s));
  CK(cudaMemsetAsync(db + p.o_status + 2 * p.n_sub + 8, 0, 16 * 8, s));
  CgArgs a;
  a.mu_out = db + p.o_muout;
  a.c_out = db + p.o_cout;
  a.max_iters = p.opt.max_iters;
  a.tol = p.opt.tol;
  a.theta = p.opt.theta;
  a.mode = 2;
  LAUNCH(PC_CG, launch_cg(p, h->ws, a, s));
  if (p.sz.sum_eval > 0) {
    LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_solve + 4], h->ws, s));
    if (d_u_eval)
      for (const auto &d : p.subs)
        if (d.nE > 0)
          CK(cudaMemcpyAsync(d_u_eval + d.eval_off * R, db + d.oU, (size_t)d.nE * R * 8, cudaMemcpyDeviceToDevice,
                             s));
  }
  if (d_r && p.n_dl > 0) CK(cudaMemcpyAsync(d_r, res, (size_t)p.n_dl * R * 8, cudaMemcpyDeviceToDevice, s));
  if (d_c) CK(cudaMemcpyAsync(d_c, db + p.o_cout, (size_t)p.sz.sum_M * R * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  int herr = 0;
  CK(cudaMemcpy(&herr, db + p.o_status + 2 * p.n_sub + 16, sizeof(int), cudaMemcpyDeviceToHost));
  return herr ? DDELM_ERR_TIMEOUT : DDELM_OK;
}

int ddelm_interface_solve(ddelm_handle *h, const double *d_b, double *d_mu_delta, ddelm_solve_info *info,
                          void *stream) {
  if (!h || !d_b || !d_mu_delta) return DDELM_ERR_INVALID_ARG;
  Plan &p = h->plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *db = dbase(h);
  const int R = p.n_rhs;
  double *mu = nullptr, *rhs = nullptr, *res = nullptr;
  cg_vectors(p, h->ws, &mu, &rhs, &res);
  if (p.n_dl == 0) return DDELM_OK;
  CK(cudaMemcpyAsync(rhs, d_b, (size_t)p.n_dl * R * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(db + p.o_status + 2 * p.n_sub + 8, 0, 16 * 8, s));
  CgArgs a;
  a.mu_out = nullptr;
  a.c_out = nullptr;
  a.max_iters = p.opt.max_iters;
  a.tol = p.opt.tol;
  a.theta = p.opt.theta;
  a.max_refine = p.opt.max_refine;
  a.mode = 3;
  LAUNCH(PC_CG, launch_cg(p, h->ws, a, s));
  CK(cudaMemcpyAsync(d_mu_delta, mu, (size_t)p.n_dl * R * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  const long long nd = p.n_dl > 0 ? p.n_dl : 1, np = p.n_pi > 0 ? p.n_pi : 1;
  double hinfo[40];
  CK(cudaMemcpy(hinfo, db + p.o_cg + 12 * nd * R + 14 * np * R + 2048 * 32 - 64, sizeof(hinfo),
                cudaMemcpyDeviceToHost));
  int herr = 0;
  CK(cudaMemcpy(&herr, db + p.o_status + 2 * p.n_sub + 16, sizeof(int), cudaMemcpyDeviceToHost));
  int rc = herr ? DDELM_ERR_TIMEOUT : DDELM_OK;
  double resmax = 0.0;
  for (int k = 0; k < R; ++k) resmax = hinfo[1 + k] > resmax ? hinfo[1 + k] : resmax;
  if (rc == DDELM_OK && int(hinfo[0]) >= p.opt.max_iters && !(resmax < p.opt.tol)) rc = DDELM_ERR_NOT_CONVERGED;
  if (info) {
    info->iterations = int(hinfo[0]);
    info->refinements = p.mixed ? int(hinfo[33]) : 0;
    info->rel_residual = resmax;
    info->ms_total = 0.0;
  }
  return rc;
}

int ddelm_backward(ddelm_handle *h, const double *d_grad_c, const double *d_grad_u, double *d_grad_f,
                   double *d_grad_g, double *h_grad_scale, ddelm_solve_info *info, void *stream) {
  if (!h) return DDELM_ERR_INVALID_ARG;
  Plan &p = h->plan;
  if (h_grad_scale && p.op == DDELM_OP_BIHARMONIC) return DDELM_ERR_UNSUPPORTED;
  if (h_grad_scale && (!h->fwd_valid || p.inv_scale == 0.0)) return DDELM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *db = dbase(h);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (info) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
  }
  const auto &G = p.setup_gemm;
  LAUNCH(PC_OTHER, launch_adjoint_init(p, h->ws, d_grad_c, d_grad_u, s));
  if (d_grad_u && p.sz.sum_eval > 0) LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_adj + 0], h->ws, s));
  LAUNCH(PC_OTHER, launch_copy_c_to_y(p, h->ws, s));
  CK(cudaMemsetAsync(db + p.o_status + 2 * p.n_sub + 8, 0, 16 * 8, s));
  CgArgs a;
  a.mu_out = nullptr;
  a.c_out = nullptr;
  a.max_iters = p.opt.max_iters;
  a.tol = p.opt.tol;
  a.theta = p.opt.theta;
  a.mode = 1;
  LAUNCH(PC_CG, launch_cg(p, h->ws, a, s));
  for (int q = 1; q <= 5; ++q) LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_adj + q], h->ws, s));
  LAUNCH(PC_OTHER, launch_adjoint_scatter(p, h->ws, d_grad_f, d_grad_g, s));
  if (h_grad_scale) {
    // dL/ds at the last solve: b-bar = S_theta^{-1} mu-bar (the adjoint solution
    // above) into the bank, the solve's mu back into the CG vector, the forward
    // y, p, a of its data recomputed; then the interface vectors (mode 4), the
    // coarse chain, and per wave the local matrices, their s-derivatives and the
    // contraction
    const long long nd = p.n_dl > 0 ? p.n_dl : 1;
    double *mu = nullptr, *rhs = nullptr, *res = nullptr;
    cg_vectors(p, h->ws, &mu, &rhs, &res);
    if (p.n_dl > 0) {
      CK(cudaMemcpyAsync(db + p.o_bank_dl + (long long)SD_BB * nd * p.n_rhs, mu, (size_t)p.n_dl * p.n_rhs * 8,
                         cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(mu, db + p.o_muout + (long long)p.n_pi * p.n_rhs, (size_t)p.n_dl * p.n_rhs * 8,
                         cudaMemcpyDeviceToDevice, s));
    }
    LAUNCH(PC_OTHER, launch_gather_rhs(p, h->ws, db + p.o_fin, db + p.o_gin, s));
    for (int q = 0; q < 4; ++q) LAUNCH(PC_GEMM, launch_gemm_phase(p, G[p.ph_solve + q], h->ws, s));
    CgArgs a4;
    a4.mu_out = nullptr;
    a4.c_out = nullptr;
    a4.max_iters = p.opt.max_iters;
    a4.tol = p.opt.tol;
    a4.theta = p.opt.theta;
    a4.mode = 4;
    LAUNCH(PC_CG, launch_cg(p, h->ws, a4, s));
    for (const auto &ph : p.sc_coarse) LAUNCH(PC_GEMM, launch_gemm_phase(p, ph, h->ws, s));
    for (int w = 0; w < p.n_waves; ++w) {
      LAUNCH(PC_FEAT, launch_scale_features(p, h->ws, w, s));
      LAUNCH(PC_OTHER, launch_scale_gather(p, h->ws, w, p.opt.theta, s));
      for (const auto &ph : p.sc_wave[w]) LAUNCH(PC_GEMM, launch_gemm_phase(p, ph, h->ws, s));
      LAUNCH(PC_OTHER, launch_scale_dots(p, h->ws, w, s));
    }
    LAUNCH(PC_OTHER, launch_scale_total(p, h->ws, p.opt.eps_rel, s));
  }
  if (info) CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  const long long nd = p.n_dl > 0 ? p.n_dl : 1, np = p.n_pi > 0 ? p.n_pi : 1;
  double it = 0.0;
  CK(cudaMemcpy(&it, db + p.o_cg + 12 * nd * p.n_rhs + 14 * np * p.n_rhs + 2048 * 32 - 64, sizeof(double),
                cudaMemcpyDeviceToHost));
  int herr = 0;
  CK(cudaMemcpy(&herr, db + p.o_status + 2 * p.n_sub + 16, sizeof(int), cudaMemcpyDeviceToHost));
  int rc = herr ? DDELM_ERR_TIMEOUT : DDELM_OK;
  if (rc == DDELM_OK && int(it) >= p.opt.max_iters) rc = DDELM_ERR_NOT_CONVERGED;
  if (h_grad_scale)
    CK(cudaMemcpy(h_grad_scale, db + p.o_gs + (long long)p.dots.size() + p.n_sub, sizeof(double),
                  cudaMemcpyDeviceToHost));
  if (info) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    info->iterations = int(it);
    info->refinements = 0;
    info->rel_residual = 0.0;
    info->ms_total = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return rc;
}

int ddelm_inspect(ddelm_handle *h, int sub, int which, double *host_out, size_t out_len) {
  if (!h || !host_out) return DDELM_ERR_INVALID_ARG;
  Plan &p = h->plan;
  double *db = dbase(h);
  if (which == 6) {
    const size_t n = (size_t)p.n_pi * p.n_pi;
    if (n > out_len) return DDELM_ERR_INVALID_ARG;
    if (n) CK(cudaMemcpy(host_out, db + p.o_Spi, n * 8, cudaMemcpyDeviceToHost));
    return DDELM_OK;
  }
  if (sub < 0 || sub >= p.n_sub) return DDELM_ERR_INVALID_ARG;
  const SubDev &d = p.subs[sub];
  long long src = -1;
  size_t n = 0;
  switch (which) {
    case 0:
    case 1:
    case 2: {
      if (!p.keep) return DDELM_ERR_UNSUPPORTED;
      long long off = p.o_keepX;
      for (int i = 0; i < sub; ++i) {
        const SubDev &e = p.subs[i];
        off += (2LL * e.m * e.M + (long long)e.nG * e.M + 31) / 32 * 32;
      }
      const long long mm = (long long)d.m * d.M;
      src = off + (which == 0 ? 0 : which == 1 ? mm : 2 * mm);
      n = which == 2 ? (size_t)d.nG * d.M : (size_t)mm;
      break;
    }
    case 3:
      src = d.oLam;
      n = (size_t)d.nG * d.nG;
      break;
    case 4:
      src = d.oPsi;
      n = (size_t)d.nG * d.nG;
      break;
    case 5:
      src = d.oPhi;
      n = (size_t)d.nDl * d.nDl;
      break;
    case 10:
      src = d.oV;
      n = (size_t)d.M * d.M;
      break;
    case 8: {  // algorithmic flops: setup GEMMs, Cholesky+inverse, solve GEMMs (no CG),
               // tensor-core flops of the MIXED setup, FP64-engine flops left in MIXED
      if (out_len < 5) return DDELM_ERR_INVALID_ARG;
      double fs = 0.0, fv = 0.0, fleft = 0.0;
      for (size_t q = 0; q < p.phase_flops.size(); ++q) {
        if ((int)q < p.ph_solve) fs += p.phase_flops[q];
        else if ((int)q < p.ph_adj) fv += p.phase_flops[q];
        if ((int)q < p.ph_solve && !(p.mixed && q < p.oz_phase.size() && p.oz_phase[q].ntile > 0))
          fleft += p.phase_flops[q];
      }
      host_out[0] = fs;
      host_out[1] = p.chol_flops;
      host_out[2] = fv;
      host_out[3] = p.oz_flops;
      host_out[4] = p.mixed ? fleft : fs;
      if (out_len >= 6) host_out[5] = p.chol_flops32;
      if (out_len >= 7) host_out[6] = p.slice_bytes;
      return DDELM_OK;
    }
    case 11: {  // tile-shape autotuner: phases timed, phases switched, their ms by the rule / as chosen
      if (out_len < 4) return DDELM_ERR_INVALID_ARG;
      host_out[0] = h->tune_phases + h->plan.tune_from_cache;
      host_out[1] = h->tune_switched;
      host_out[2] = h->tune_ms_rule;
      host_out[3] = h->tune_ms_chosen;
      for (size_t k = 0; k < h->tune_log.size() && 4 + k < out_len; ++k) host_out[4 + k] = h->tune_log[k];
      return DDELM_OK;
    }
    case 9: {
      if (out_len < 4) return DDELM_ERR_INVALID_ARG;
      host_out[0] = p.scheme;
      host_out[1] = p.n_pass;
      host_out[2] = p.n_waves;
      host_out[3] = p.wave;
      if (out_len >= 6) {
        host_out[4] = h->setup_exec ? 1.0 : 0.0;
        host_out[5] = h->solve_exec ? 1.0 : 0.0;
      }
      return DDELM_OK;
    }
    case 7: {
      if (out_len < 4) return DDELM_ERR_INVALID_ARG;
      host_out[0] = d.m;
      host_out[1] = d.M;
      host_out[2] = d.nG;
      host_out[3] = d.nDl;
      return DDELM_OK;
    }
    default:
      return DDELM_ERR_INVALID_ARG;
  }
  if (n > out_len) return DDELM_ERR_INVALID_ARG;
  if (n) CK(cudaMemcpy(host_out, db + src, n * 8, cudaMemcpyDeviceToHost));
  return DDELM_OK;
}

int ddelm_profile(ddelm_handle *h, int enable, int reset, double *ms, long long *launches) {
  if (!h) return DDELM_ERR_INVALID_ARG;
  for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
    CK(cudaEventSynchronize(h->ev[k + 1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->ev[k], h->ev[k + 1]));
    h->prof_ms[h->ev_cls[k]] += t;
    h->prof_n[h->ev_cls[k]] += h->ev_kernels[k];
  }
  h->ev_used = 0;
  for (int c = 0; c < DDELM_PROF_CLASSES; ++c) {
    if (ms) ms[c] = h->prof_ms[c];
    if (launches) launches[c] = h->prof_n[c];
    if (reset) {
      h->prof_ms[c] = 0.0;
      h->prof_n[c] = 0;
    }
  }
  h->prof = enable != 0;
  return DDELM_OK;
}

void ddelm_destroy(ddelm_handle *h) {
  if (!h) return;
  for (auto e : h->ev) cudaEventDestroy(e);
  if (h->setup_exec) cudaGraphExecDestroy(h->setup_exec);
  if (h->solve_exec) cudaGraphExecDestroy(h->solve_exec);
  delete h;
}

const char *ddelm_last_error(void) { return ddelm::g_last_error; }

const char *ddelm_status_string(int status) {
  switch (status) {
    case DDELM_OK:
      return "ok";
    case DDELM_ERR_INVALID_ARG:
      return "invalid argument";
    case DDELM_ERR_RANK_DEFICIENT:
      return "a local factorisation failed (a non-positive pivot, or a Gram too far from I for the series)";
    case DDELM_ERR_NOT_CONVERGED:
      return "CG reached max_iters before the tolerance";
    case DDELM_ERR_CUDA:
      return "CUDA runtime error";
    case DDELM_ERR_TIMEOUT:
      return "a device grid barrier timed out";
    case DDELM_ERR_UNSUPPORTED:
      return "unsupported option or call";
    default:
      return "unknown status";
  }
}

}  // extern "C"
