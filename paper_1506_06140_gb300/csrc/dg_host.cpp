// libdg host side: the C ABI of include/dg.h.  Builds the mesh and face
// tables, the quadrature tables, and the per-step stage program; launches the
// kernels of dg_kernels.cuh on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "dg.h"
#include "dg_internal.h"

using namespace dgi;

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------------------
// 1D rules on [-1,1] (Appendices B and C), computed by Newton iteration.

double leg_p(int n, double x, double* dp) {
  // value and derivative of P_n by the three-term recurrence
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *dp = 0.0; return 1.0; }
  for (int m = 1; m < n; ++m) {
    const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    const double d2 = d0 + (2.0 * m + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *dp = d1;
  return p1;
}

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int q = 0; q < n; ++q) {
    // Lether's approximation of root q (largest first), then Newton
    double r = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) *
               std::cos(M_PI * (4.0 * (q + 1) - 1.0) / (4.0 * n + 2.0));
    double d = 0.0;
    for (int it = 0; it < 64; ++it) {
      const double p = leg_p(n, r, &d);
      const double step = p / d;
      r -= step;
      if (std::fabs(step) <= 1e-16) break;
    }
    leg_p(n, r, &d);
    x[n - 1 - q] = r;
    w[n - 1 - q] = 2.0 / ((1.0 - r * r) * d * d);
  }
}

void lobatto_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  x[0] = -1.0;
  x[n - 1] = 1.0;
  const int m = n - 1;
  double sum = 0.0;
  for (int q = 1; q < n - 1; ++q) {
    double r = -std::cos(M_PI * q / m);
    for (int it = 0; it < 64; ++it) {
      double d;
      const double p = leg_p(m, r, &d);
      // Newton on P'_m using P''_m = (2 r P'_m - m (m+1) P_m) / (1 - r^2)
      const double d2 = (2.0 * r * d - m * (m + 1.0) * p) / (1.0 - r * r);
      const double step = d / d2;
      r -= step;
      if (std::fabs(step) <= 1e-16) break;
    }
    double d;
    const double p = leg_p(m, r, &d);
    x[q] = r;
    w[q] = 2.0 / (n * (n - 1.0) * p * p);
    sum += w[q];
  }
  w[0] = w[n - 1] = 0.5 * (2.0 - sum);
}

// ---------------------------------------------------------------------------
// Step program: the Butcher tableau (Appendix D) rewritten as a sequence of
// stages, each evaluating dW/dt at one stored state and forming at most three
// linear combinations of stored arrays and the new derivative.

struct Tab {
  int s = 0;
  std::vector<double> A, b;
};

Tab butcher(int order) {
  Tab t;
  if (order == 1) { t.s = 1; t.A = {0}; t.b = {1}; }
  else if (order == 2) { t.s = 2; t.A = {0, 0, 1, 0}; t.b = {0.5, 0.5}; }
  else if (order == 3) {
    t.s = 3;
    t.A = {0, 0, 0, 1, 0, 0, 0.25, 0.25, 0};
    t.b = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  } else {
    // SSP RK(5,4), Table RK_4
    t.s = 5;
    t.A.assign(25, 0.0);
    const double a[5][5] = {{0, 0, 0, 0, 0},
                            {0.39175222700392, 0, 0, 0, 0},
                            {0.21766909633821, 0.36841059262959, 0, 0, 0},
                            {0.08269208670950, 0.13995850206999, 0.25189177424738, 0, 0},
                            {0.06796628370320, 0.11503469844438, 0.20703489864929,
                             0.54497475021237, 0}};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) t.A[i * 5 + j] = a[i][j];
    t.b = {0.14681187618661, 0.24848290924556, 0.10425883036650, 0.27443890091960,
           0.22600748319395};
  }
  return t;
}

struct Op {
  int in_reg = 0;                 // state whose dW/dt is evaluated
  int n_in = 0, n_out = 0;
  int in[MAX_IN] = {0, 0, 0, 0};
  int out[MAX_OUT] = {0, 0, 0};
  double C[MAX_OUT][MAX_IN] = {};
  double ck[MAX_OUT] = {};
  int lim_src = -1, lim_dst = -1; // limiter pass after the stage (virtual registers)
};

struct Program {
  std::vector<Op> ops;
  int n_phys = 0;                 // scratch registers needed (register 0 is the caller's W)
};

// least squares: min |sum_r lam_r V_r - t|, returns residual norm
double lsq(const std::vector<std::vector<double>>& V, const std::vector<double>& t,
           std::vector<double>& lam) {
  const int n = (int)V.size(), m = (int)t.size();
  std::vector<double> G(n * n, 0.0), r(n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < m; ++k) G[i * n + j] += V[i][k] * V[j][k];
    for (int k = 0; k < m; ++k) r[i] += V[i][k] * t[k];
  }
  // Gaussian elimination with partial pivoting
  std::vector<int> piv(n);
  for (int i = 0; i < n; ++i) piv[i] = i;
  for (int c = 0; c < n; ++c) {
    int best = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(G[i * n + c]) > std::fabs(G[best * n + c])) best = i;
    if (std::fabs(G[best * n + c]) < 1e-300) return 1e300;
    if (best != c) {
      for (int j = 0; j < n; ++j) std::swap(G[c * n + j], G[best * n + j]);
      std::swap(r[c], r[best]);
    }
    for (int i = c + 1; i < n; ++i) {
      const double f = G[i * n + c] / G[c * n + c];
      for (int j = c; j < n; ++j) G[i * n + j] -= f * G[c * n + j];
      r[i] -= f * r[c];
    }
  }
  lam.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= G[i * n + j] * lam[j];
    lam[i] = s / G[i * n + i];
  }
  double res = 0.0;
  for (int k = 0; k < m; ++k) {
    double s = -t[k];
    for (int i = 0; i < n; ++i) s += lam[i] * V[i][k];
    res += s * s;
  }
  return std::sqrt(res);
}

// Express target t (coordinates: [alpha, k_0..k_{s-1}], the k_i entry
// already removed) with as few of the candidate registers as possible.
bool represent(const std::vector<int>& cand, const std::map<int, std::vector<double>>& content,
               const std::vector<double>& t, std::vector<int>& used, std::vector<double>& lam) {
  double tn = 0.0;
  for (double x : t) tn += x * x;
  tn = std::sqrt(tn);
  if (tn == 0.0) { used.clear(); lam.clear(); return true; }
  const int nc = (int)cand.size();
  for (int size = 1; size <= std::min(nc, MAX_IN); ++size) {
    std::vector<int> idx(size);
    for (int i = 0; i < size; ++i) idx[i] = i;
    while (true) {
      std::vector<std::vector<double>> V;
      for (int i : idx) V.push_back(content.at(cand[i]));
      std::vector<double> l;
      const double res = lsq(V, t, l);
      if (res <= 1e-9 * (tn + 1.0)) {
        used.clear();
        for (int i : idx) used.push_back(cand[i]);
        lam = l;
        return true;
      }
      int p = size - 1;
      while (p >= 0 && idx[p] == nc - size + p) --p;
      if (p < 0) break;
      ++idx[p];
      for (int i = p + 1; i < size; ++i) idx[i] = idx[i - 1] + 1;
    }
  }
  return false;
}

// Builds the stage program of one step.  Without limiting the stage states
// themselves serve as registers (U_i = w + dt sum_j a_ij k_j), so every
// stage reads at most the stage state, w and one earlier state.  With
// limiting, the stage states are limited and carry no such identity; the
// program keeps accumulators of dt * (combinations of k_j) instead, chosen as
// a basis of the combinations later stages and the final update still need.
bool build_program(int order, bool limited, Program& P, std::string& err) {
  const Tab tb = butcher(order);
  const int s = tb.s;
  const int dimv = 1 + s;  // coordinates: alpha (coefficient of w), k_0..k_{s-1}
  std::map<int, std::vector<double>> content;  // virtual register -> coordinates
  content[0] = std::vector<double>(dimv, 0.0);
  content[0][0] = 1.0;
  int next_vreg = 1;
  int cur = 0;  // virtual register holding the current stage state
  std::vector<int> accs;  // accumulator registers (limited mode)
  std::vector<Op> ops;
  for (int i = 0; i < s; ++i) {
    Op op;
    op.in_reg = cur;
    const bool last = (i == s - 1);
    // targets: next stage state (or final state), then accumulators
    std::vector<std::vector<double>> targets;
    std::vector<double> t0(dimv, 0.0);
    t0[0] = 1.0;
    for (int j = 0; j <= i; ++j) t0[1 + j] = last ? tb.b[j] : tb.A[(i + 1) * s + j];
    if (last)
      for (int j = 0; j < s; ++j) t0[1 + j] = tb.b[j];
    targets.push_back(t0);
    std::vector<int> new_accs;
    if (limited && !last) {
      // combinations of k_0..k_i still needed after this stage
      std::vector<std::vector<double>> needs;
      for (int m = i + 2; m < s; ++m) {
        std::vector<double> v(dimv, 0.0);
        for (int j = 0; j <= i; ++j) v[1 + j] = tb.A[m * s + j];
        needs.push_back(v);
      }
      {
        std::vector<double> v(dimv, 0.0);
        for (int j = 0; j <= i; ++j) v[1 + j] = tb.b[j];
        needs.push_back(v);
      }
      std::vector<std::vector<double>> basis;
      for (auto& v : needs) {
        std::vector<double> l;
        bool dep = false;
        if (!basis.empty()) {
          double vn = 0.0;
          for (double x : v) vn += x * x;
          dep = lsq(basis, v, l) <= 1e-9 * (std::sqrt(vn) + 1.0);
        }
        bool zero = true;
        for (double x : v) zero = zero && x == 0.0;
        if (!dep && !zero) basis.push_back(v);
      }
      for (auto& v : basis) {
        targets.push_back(v);
        const int r = next_vreg++;
        content[r] = v;
        new_accs.push_back(r);
      }
    }
    // candidate inputs
    std::vector<int> cand;
    if (!limited) {
      cand.push_back(cur);
      if (cur != 0) cand.push_back(0);
      for (auto& kv : content)
        if (kv.first != cur && kv.first != 0 &&
            std::find(new_accs.begin(), new_accs.end(), kv.first) == new_accs.end())
          cand.push_back(kv.first);
    } else {
      cand.push_back(0);
      for (int r : accs) cand.push_back(r);
    }
    std::vector<int> ins;
    std::vector<std::vector<double>> coefs;
    for (size_t o = 0; o < targets.size(); ++o) {
      std::vector<double> t = targets[o];
      const double cki = t[1 + i];
      t[1 + i] = 0.0;
      std::vector<int> used;
      std::vector<double> lam;
      if (!represent(cand, content, t, used, lam)) {
        err = "internal: Runge-Kutta stage program has no representation";
        return false;
      }
      op.ck[o] = cki;
      for (size_t u = 0; u < used.size(); ++u) {
        auto it = std::find(ins.begin(), ins.end(), used[u]);
        int slot;
        if (it == ins.end()) {
          ins.push_back(used[u]);
          slot = (int)ins.size() - 1;
        } else {
          slot = (int)(it - ins.begin());
        }
        if (slot >= MAX_IN) { err = "internal: too many stage inputs"; return false; }
        op.C[o][slot] = lam[u];
      }
    }
    op.n_in = (int)ins.size();
    for (int r = 0; r < op.n_in; ++r) op.in[r] = ins[r];
    op.n_out = (int)targets.size();
    if (op.n_out > MAX_OUT) { err = "internal: too many stage outputs"; return false; }
    // output registers
    int stage_out;
    if (!limited) {
      stage_out = last ? 0 : next_vreg++;
      if (!last) content[stage_out] = targets[0];
      op.out[0] = stage_out;
      cur = stage_out;
    } else {
      stage_out = next_vreg++;  // unlimited value, limited into lim_dst
      op.out[0] = stage_out;
      const int dst = last ? 0 : next_vreg++;
      op.lim_src = stage_out;
      op.lim_dst = dst;
      cur = dst;
    }
    for (size_t o = 1; o < targets.size(); ++o) op.out[o] = new_accs[o - 1];
    if (limited) accs = new_accs;
    ops.push_back(op);
  }
  // register allocation: virtual -> physical by live ranges
  const int nops = (int)ops.size();
  std::map<int, int> def, last_use;
  for (int i = 0; i < nops; ++i) {
    const Op& op = ops[i];
    auto use = [&](int r) { last_use[r] = std::max(last_use.count(r) ? last_use[r] : i, i); };
    use(op.in_reg);
    for (int r = 0; r < op.n_in; ++r) use(op.in[r]);
    for (int o = 0; o < op.n_out; ++o) if (!def.count(op.out[o])) def[op.out[o]] = i;
    if (op.lim_src >= 0) { use(op.lim_src); if (!def.count(op.lim_dst)) def[op.lim_dst] = i; }
  }
  std::map<int, int> phys;
  phys[0] = 0;
  std::vector<int> busy_until;  // per physical scratch register (1-based index = p)
  for (int i = 0; i < nops; ++i) {
    std::vector<int> defs;
    for (int o = 0; o < ops[i].n_out; ++o) defs.push_back(ops[i].out[o]);
    if (ops[i].lim_dst >= 0) defs.push_back(ops[i].lim_dst);
    for (int r : defs) {
      if (phys.count(r)) continue;
      const int end = last_use.count(r) ? last_use[r] : i;
      int p = -1;
      for (size_t j = 0; j < busy_until.size(); ++j)
        if (busy_until[j] < i) { p = (int)j; break; }
      if (p < 0) { busy_until.push_back(0); p = (int)busy_until.size() - 1; }
      busy_until[p] = std::max(end, i);
      phys[r] = p + 1;
    }
  }
  for (auto& op : ops) {
    op.in_reg = phys.at(op.in_reg);
    for (int r = 0; r < op.n_in; ++r) op.in[r] = phys.at(op.in[r]);
    for (int o = 0; o < op.n_out; ++o) op.out[o] = phys.at(op.out[o]);
    if (op.lim_src >= 0) { op.lim_src = phys.at(op.lim_src); op.lim_dst = phys.at(op.lim_dst); }
  }
  P.ops = ops;
  P.n_phys = (int)busy_until.size();
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------

struct dg_handle {
  int dim = 2, k = 1, prec = DG_FP64, nv = 4, N = 3;
  double gamma = 1.4;
  dg_options opt{};
  const KernelSet* ks = nullptr;
  size_t esize = 8;  // bytes per state element
  // host mesh tables
  int ncells = 0, nfaces = 0, nnodes = 0;
  std::vector<int32_t> nbr, coord, node_children, fm, fp, sface;
  std::vector<int8_t> level;
  std::vector<uint8_t> finfo, scoarse;
  MeshDev md;
  double volume = 1.0;
  // device memory
  std::vector<void*> allocs;
  void* tab = nullptr;
  double* tab64 = nullptr;
  Tab1D<double> tab1d64{};
  float* tab32 = nullptr;    // the tables in FP32 (positivity precheck)
  void* F = nullptr;
  std::vector<void*> regs;   // scratch state registers 1..n
  bool use_tc = false;       // tensor-core cell kernel (DG_FP32_TC, DG_MIXED_TC)
  int tc_hook = 0;           // dg_test_force_timeout: armed for the next tensor-core cell launch
  const MixedSet* ms = nullptr;  // FP32 perturbation-form stage kernels (DG_MIXED)
  Tab1D<float> tab1d32{};
  float* Gm = nullptr;       // DG_MIXED face fluxes minus the minus cell's reference flux
  float* Dm = nullptr;       // DG_MIXED reference flux differences per face
  bool delta = false;        // DG_MIXED with FP32 delta registers (unlimited programs)
  unsigned long long* lim_counts = nullptr;  // [3] cells changed by the slope / positivity limiter,
                                             // cells examined by the FP64 positivity pass
  int* lim_queue = nullptr;  // [ncells + 1]: the positivity pass's cells, then their number
  float* Wf = nullptr;       // delta mode: FP32 split of W within a step [NV][N][ncells]
  float* Wlo = nullptr;      //             and the rest of weight 0 [NV][ncells]
  int cell_tile = 0, face_tile = 0;  // stage-kernel tiles (0: the kernels' defaults)
  bool use_direct = false;   // one-thread-per-cell FP32 cell kernel
  bool use_x2 = false;       // packed-pair FP32 cell kernel (two variables per thread)
  int pdl = 1;               // stage kernels launched as programmatic dependents (dg_set_overlap)
  bool use_fused = false;    // fused face + cell kernel (face tile 0)
  std::vector<unsigned char> dtab;  // its tables (host copy, passed by value at launch)
  void* tcB = nullptr;       // its B operands
  double* scal = nullptr;    // dt per problem [nprob]
  unsigned long long* dt_bits = nullptr;  // per-problem max signal speed [nprob] (zero between launches)
  unsigned int* dt_done = nullptr;        // blocks of the dt kernel done (zero between launches)
  // ensembles
  int nprob = 1;
  std::vector<int32_t> prob;
  std::vector<double> dx_prob, lo_prob;
  void* pre_prob = nullptr;       // [nprob] 2^(1-d)/dx in the handle precision
  double* inv_dx_prob = nullptr;  // [nprob]
  double* partial = nullptr;
  int* status = nullptr;
  Program prog_step;         // limited as configured
  Program prog_free;         // unlimited (adjoint recomputation)
  cudaStream_t cap_stream = nullptr;
  // dg_advance / dg_advance_dt graphs per (W, n_steps, dt history, fixed dt; 0 = CFL)
  std::map<std::tuple<void*, int, void*, double>, cudaGraphExec_t> graphs;
  std::vector<cudaGraph_t> graph_defs;
  // dg_advance as one persistent kernel: mode, plans per (W, dt history)
  // with their largest phase's block count, the grid barrier's words
  int advance_mode = DG_ADVANCE_GRAPH;
  std::map<std::pair<void*, void*>, std::pair<void*, int>> plans;
  unsigned* bar = nullptr;
  std::string err;
  std::mutex mu;
  // adjoint work arrays (allocated by the first dg_rk_step_adjoint call)
  std::vector<void*> adj;
  void* FG = nullptr;
  // dynamic adaptation (single problems): base grid, the base maps of the
  // current mesh (slot cur) and of the marked next mesh (slot 1 - cur)
  BaseGrid bg;
  std::vector<int32_t> base_first_host, base_node_host;  // of the mesh built at creation
  int32_t* base_first[2] = {nullptr, nullptr};  // [nbase + 1]
  int32_t* base_node[2] = {nullptr, nullptr};   // [nbase]
  int cur = 0;
  uint8_t* adapt_crit = nullptr;   // [nbase] criterion
  uint8_t* adapt_ref = nullptr;    // [nbase] new refinement
  int32_t* adapt_cnt = nullptr;    // [nbase] cells per base cell
  int32_t* adapt_info = nullptr;   // [1] base cells whose refinement changes
  int32_t* scan_work = nullptr;
  size_t scan_work_cap = 0;
  int32_t* face_cnt = nullptr;     // regrid face counts and their prefix sums
  int32_t* face_off = nullptr;
  size_t face_cnt_cap = 0;
  bool mark_pending = false;
  int64_t next_cells = 0, next_nodes = 0;
  size_t cap_cells = 0, cap_faces = 0, cap_nodes = 0;  // capacity of the mesh-sized buffers
  bool tables_on_device = false;   // host mirrors are stale after a regrid
  // gravity: external acceleration [dim][Q][ncells] in the state precision
  void* accel = nullptr;
  bool accel_stale = false;  // dropped by a regrid: set again before stepping
  // instrumentation
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks;  // (kind, index of the start event)
  // dg_advance while profiling: graphs recorded with their event pairs as
  // event-record nodes (each with its own events), and the device times of
  // their replays summed per kernel kind
  struct ProfGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<std::pair<int, size_t>> marks;
  };
  std::map<std::tuple<void*, int, void*, double>, ProfGraph> pgraphs;
  double prof_ms[DG_KERNEL_KINDS] = {};
  int prof_n[DG_KERNEL_KINDS] = {};
};

namespace {

int fail(dg_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(dg_handle* h, cudaError_t e, const char* what) {
  return fail(h, DG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DG_CUDA(h, call)                                       \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return cuda_fail((h), e__, #call); \
  } while (0)

// Runs one kernel launcher; with profiling on, brackets it by two events.
template <typename F>
cudaError_t timed(dg_handle* h, int kind, cudaStream_t s, F&& launch) {
  if (!h->profiling) return launch();
  while (h->ev_pool.size() < h->ev_used + 2) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    h->ev_pool.push_back(e);
  }
  const size_t i0 = h->ev_used;
  h->ev_used += 2;
  // inside a stream capture the records are external: they become
  // event-record nodes of the graph (recorded at every replay)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(s, &cs);
  if (r != cudaSuccess) return r;
  const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  r = cudaEventRecordWithFlags(h->ev_pool[i0], s, flags);
  if (r != cudaSuccess) return r;
  r = launch();
  if (r != cudaSuccess) return r;
  r = cudaEventRecordWithFlags(h->ev_pool[i0 + 1], s, flags);
  h->ev_marks.push_back({kind, i0});
  return r;
}

template <typename T>
int upload(dg_handle* h, const std::vector<T>& v, const T** out) {
  if (v.empty()) { *out = nullptr; return DG_OK; }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, v.size() * sizeof(T));
  if (e != cudaSuccess) return fail(h, DG_ERR_OOM, "cudaMalloc of a mesh table failed");
  h->allocs.push_back(p);
  e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy");
  *out = static_cast<const T*>(p);
  return DG_OK;
}

void dfree(dg_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) h->allocs.erase(it);
  cudaFree(p);
}

int dalloc(dg_handle* h, size_t bytes, void** out) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, DG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  h->allocs.push_back(p);
  *out = p;
  return DG_OK;
}

// Mesh tables by index arithmetic over the base grid: every base cell owns
// one cell (unrefined) or 2^dim consecutive children (refined).
int build_mesh(dg_handle* h, const dg_mesh_desc* m) {
  const int d = m->dim;
  int n[3] = {1, 1, 1};
  int bc[3] = {DG_BC_PERIODIC, DG_BC_PERIODIC, DG_BC_PERIODIC};
  for (int a = 0; a < d; ++a) {
    n[a] = m->n[a];
    bc[a] = m->bc[a];
    if (n[a] < 1) return fail(h, DG_ERR_ARG, "mesh: n must be >= 1");
    if (bc[a] != DG_BC_PERIODIC && bc[a] != DG_BC_TRANSMISSIVE)
      return fail(h, DG_ERR_ARG, "mesh: unknown boundary condition");
    if (!(m->hi[a] > m->lo[a])) return fail(h, DG_ERR_ARG, "mesh: hi must exceed lo");
  }
  const double dx0 = (m->hi[0] - m->lo[0]) / n[0];
  for (int a = 1; a < d; ++a)
    if (std::fabs((m->hi[a] - m->lo[a]) / n[a] - dx0) > 1e-12 * dx0)
      return fail(h, DG_ERR_ARG, "mesh: cells must be cubical (equal edge length on all axes)");
  const int64_t nbase64 = (int64_t)n[0] * n[1] * n[2];
  if (nbase64 > (1LL << 28)) return fail(h, DG_ERR_ARG, "mesh: too many base cells");
  const int nbase = (int)nbase64;
  std::vector<uint8_t> refined(nbase, 0);
  if (m->n_refine_boxes > 0 && !m->refine_boxes) return fail(h, DG_ERR_ARG, "mesh: refine_boxes is NULL");
  for (int b = 0; b < m->n_refine_boxes; ++b) {
    const int32_t* bx = m->refine_boxes + 2 * d * b;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      lo[a] = std::max(0, (int)bx[a]);
      hi[a] = std::min(n[a] - 1, (int)bx[d + a]);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) refined[x + n[0] * (y + n[1] * z)] = 1;
  }
  const int nch = 1 << d;
  std::vector<int32_t> first(nbase + 1, 0), node_of(nbase, -1);
  int nn = 0;
  for (int b = 0; b < nbase; ++b) {
    first[b + 1] = first[b] + (refined[b] ? nch : 1);
    if (refined[b]) node_of[b] = nn++;
  }
  const int nc = first[nbase];
  h->ncells = nc;
  h->nnodes = nn;
  h->bg.dim = d;
  h->bg.nbase = nbase;
  for (int a = 0; a < 3; ++a) {
    h->bg.n[a] = n[a];
    h->bg.periodic[a] = a < d ? (bc[a] == DG_BC_PERIODIC) : 1;
  }
  h->base_first_host = first;
  h->base_node_host = node_of;
  h->level.assign(nc, 0);
  h->coord.assign((size_t)3 * nc, 0);
  h->node_children.assign((size_t)nn * nch, 0);
  for (int b = 0; b < nbase; ++b) {
    const int bx = b % n[0], by = (b / n[0]) % n[1], bz = b / (n[0] * n[1]);
    if (!refined[b]) {
      const int c = first[b];
      h->coord[c] = bx; h->coord[nc + c] = by; h->coord[2 * nc + c] = bz;
    } else {
      for (int ch = 0; ch < nch; ++ch) {
        const int c = first[b] + ch;
        h->level[c] = 1;
        h->coord[c] = 2 * bx + (ch & 1);
        h->coord[nc + c] = 2 * by + ((ch >> 1) & 1);
        h->coord[2 * nc + c] = d == 3 ? 2 * bz + ((ch >> 2) & 1) : 0;
        h->node_children[(size_t)node_of[b] * nch + ch] = c;
      }
    }
  }
  // neighbour table
  h->nbr.assign((size_t)2 * d * nc, -1);
  for (int c = 0; c < nc; ++c) {
    const int l = h->level[c];
    for (int a = 0; a < d; ++a)
      for (int s = 0; s < 2; ++s) {
        int p[3] = {h->coord[c], h->coord[nc + c], h->coord[2 * nc + c]};
        p[a] += s ? 1 : -1;
        const int ext = n[a] << l;
        if (p[a] < 0 || p[a] >= ext) {
          if (bc[a] != DG_BC_PERIODIC) continue;  // stays -1
          p[a] = (p[a] + ext) % ext;
        }
        const int b = (p[0] >> l) + n[0] * ((p[1] >> l) + n[1] * (p[2] >> l));
        int32_t v;
        if (l == 0) {
          v = refined[b] ? -(node_of[b] + 2) : first[b];
        } else {
          v = refined[b] ? first[b] + ((p[0] & 1) | ((p[1] & 1) << 1) | ((p[2] & 1) << 2)) : first[b];
        }
        h->nbr[(size_t)(2 * a + s) * nc + c] = v;
      }
  }
  // face entries: conforming faces and boundary faces by direction in cell
  // order (so a warp of faces maps to consecutive cells), then the hanging
  // sub-faces grouped per coarse side in quadrant order
  h->fm.clear(); h->fp.clear(); h->finfo.clear();
  h->sface.assign((size_t)2 * d * nc, -1);
  h->scoarse.assign(nc, 0);
  auto add_face = [&](int cm, int cp, int dir, int vm, int vp) {
    h->fm.push_back(cm); h->fp.push_back(cp);
    h->finfo.push_back((uint8_t)(dir | (vm << 2) | (vp << 5)));
    return (int)h->fm.size() - 1;
  };
  for (int a = 0; a < d; ++a)
    for (int c = 0; c < nc; ++c) {
      const int up = h->nbr[(size_t)(2 * a + 1) * nc + c];
      if (up == -1) {
        h->sface[(size_t)(2 * a + 1) * nc + c] = add_face(c, -1, a, 0, 0);
      } else if (up >= 0 && h->level[up] == h->level[c]) {
        const int f = add_face(c, up, a, 0, 0);
        h->sface[(size_t)(2 * a + 1) * nc + c] = f;
        h->sface[(size_t)(2 * a + 0) * nc + up] = f;
      }
      const int dn = h->nbr[(size_t)(2 * a + 0) * nc + c];
      if (dn == -1) h->sface[(size_t)(2 * a + 0) * nc + c] = add_face(-1, c, a, 0, 0);
    }
  const int nsub = 1 << (d - 1);
  for (int a = 0; a < d; ++a)
    for (int c = 0; c < nc; ++c)
      for (int s = 0; s < 2; ++s) {
        const int nb = h->nbr[(size_t)(2 * a + s) * nc + c];
        if (nb > -2) continue;
        // coarse cell c, finer node on side s: its children touching the face
        const int node = -(nb + 2);
        h->scoarse[c] |= (uint8_t)(1u << (2 * a + s));
        for (int quad = 0; quad < nsub; ++quad) {
          int ch = s ? 0 : (1 << a);  // child bit along a: adjacent layer of the node
          int t = 0;
          for (int b = 0; b < d; ++b) {
            if (b == a) continue;
            if ((quad >> t) & 1) ch |= 1 << b;
            ++t;
          }
          const int fine = h->node_children[(size_t)node * nch + ch];
          const int f = s ? add_face(c, fine, a, 1 + quad, 0) : add_face(fine, c, a, 0, 1 + quad);
          if (quad == 0) h->sface[(size_t)(2 * a + s) * nc + c] = f;
          h->sface[(size_t)(2 * a + (1 - s)) * nc + fine] = f;
        }
      }
  h->nfaces = (int)h->fm.size();
  for (size_t i = 0; i < h->sface.size(); ++i)
    if (h->sface[i] < 0) return fail(h, DG_ERR_ARG, "internal: a cell side has no face");
  h->volume = 1.0;
  for (int a = 0; a < d; ++a) h->volume *= m->hi[a] - m->lo[a];
  h->md.ncells = nc;
  h->md.nfaces = h->nfaces;
  h->md.nnodes = nn;
  h->md.dx0 = dx0;
  for (int a = 0; a < 3; ++a) {
    h->md.lo[a] = a < d ? m->lo[a] : 0.0;
    h->md.n[a] = n[a];
  }
  return DG_OK;
}

// Concatenates independent uniform problems into one cell list: problem p
// owns a contiguous range of cells, faces and table entries; indices are
// shifted by the range offsets.
int build_batch(dg_handle* h, const dg_mesh_desc* meshes, int nprob) {
  std::vector<dg_handle*> parts;
  struct Guard {
    std::vector<dg_handle*>& v;
    ~Guard() { for (auto* p : v) delete p; }
  } guard{parts};
  int nc = 0, nf = 0, nn = 0;
  for (int p = 0; p < nprob; ++p) {
    if (meshes[p].dim != meshes[0].dim)
      return fail(h, DG_ERR_ARG, "dg_create_batch: all problems need the same dim");
    if (meshes[p].n_refine_boxes != 0)
      return fail(h, DG_ERR_UNSUPPORTED, "dg_create_batch: problems must be uniform meshes");
    auto* t = new dg_handle();
    parts.push_back(t);
    const int r = build_mesh(t, &meshes[p]);
    if (r != DG_OK) return fail(h, r, "dg_create_batch: problem " + std::to_string(p) + ": " + t->err);
    if ((int64_t)nc + t->ncells > (1LL << 30)) return fail(h, DG_ERR_ARG, "dg_create_batch: too many cells");
    nc += t->ncells;
    nf += t->nfaces;
    nn += t->nnodes;
  }
  const int d = meshes[0].dim;
  h->ncells = nc;
  h->nfaces = nf;
  h->nnodes = nn;
  h->nprob = nprob;
  h->level.assign(nc, 0);
  h->coord.assign((size_t)3 * nc, 0);
  h->nbr.assign((size_t)2 * d * nc, -1);
  h->sface.assign((size_t)2 * d * nc, -1);
  h->scoarse.assign(nc, 0);
  h->prob.assign(nc, 0);
  h->fm.clear(); h->fp.clear(); h->finfo.clear();
  h->node_children.clear();
  h->dx_prob.assign(nprob, 0.0);
  h->lo_prob.assign((size_t)3 * nprob, 0.0);
  h->volume = 0.0;
  int c0 = 0;
  for (int p = 0; p < nprob; ++p) {
    const dg_handle* t = parts[p];
    const int tc = t->ncells;
    const int f0 = (int)h->fm.size();
    for (int c = 0; c < tc; ++c) {
      h->level[c0 + c] = t->level[c];
      h->prob[c0 + c] = p;
      h->scoarse[c0 + c] = t->scoarse[c];
      for (int a = 0; a < 3; ++a) h->coord[(size_t)a * nc + c0 + c] = t->coord[(size_t)a * tc + c];
      for (int sd = 0; sd < 2 * d; ++sd) {
        const int32_t v = t->nbr[(size_t)sd * tc + c];
        h->nbr[(size_t)sd * nc + c0 + c] = v >= 0 ? v + c0 : v;
        h->sface[(size_t)sd * nc + c0 + c] = t->sface[(size_t)sd * tc + c] + f0;
      }
    }
    for (size_t f = 0; f < t->fm.size(); ++f) {
      h->fm.push_back(t->fm[f] >= 0 ? t->fm[f] + c0 : -1);
      h->fp.push_back(t->fp[f] >= 0 ? t->fp[f] + c0 : -1);
      h->finfo.push_back(t->finfo[f]);
    }
    h->dx_prob[p] = t->md.dx0;
    for (int a = 0; a < 3; ++a) h->lo_prob[3 * p + a] = t->md.lo[a];
    h->volume += t->volume;
    c0 += tc;
  }
  h->md = parts[0]->md;
  h->md.ncells = nc;
  h->md.nfaces = nf;
  h->md.nnodes = nn;
  h->md.nprob = nprob;
  return DG_OK;
}

// ---- dynamic adaptation: buffers ----

template <typename T>
int realloc_buf(dg_handle* h, T*& ptr, size_t bytes) {
  dfree(h, const_cast<void*>(static_cast<const void*>(ptr)));
  ptr = nullptr;
  void* q = nullptr;
  const int r = dalloc(h, bytes, &q);
  if (r != DG_OK) return r;
  ptr = static_cast<T*>(q);
  return DG_OK;
}

// Mesh-sized buffers for at least nc cells, nf faces and nn nodes (a negative
// count leaves that class alone).  A class that does not fit is released and
// allocated anew with a quarter of headroom; contents are not kept (the
// caller rewrites every table).  cudaFree waits for the device.
int ensure_capacity(dg_handle* h, int64_t nc, int64_t nf, int64_t nn) {
  const int d = h->dim, nch = 1 << d;
  auto grown = [](int64_t need, int64_t limit) { return std::min<int64_t>(limit, need + need / 4 + 64); };
  int r;
  if (nc > (int64_t)h->cap_cells) {
    const size_t cap = (size_t)grown(nc, (int64_t)h->bg.nbase * nch);
    MeshDev& m = h->md;
    if ((r = realloc_buf(h, m.level, cap)) != DG_OK) return r;
    if ((r = realloc_buf(h, m.coord, 3 * cap * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, m.nbr, 2 * d * cap * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, m.sface, 2 * d * cap * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, m.scoarse, cap)) != DG_OK) return r;
    for (auto& reg : h->regs)
      if ((r = realloc_buf(h, reg, (size_t)h->nv * h->N * cap * h->esize)) != DG_OK) return r;
    if ((r = realloc_buf(h, h->partial, ((cap + 255) / 256 + 1) * 8 * sizeof(double))) != DG_OK) return r;
    if ((r = realloc_buf(h, h->lim_queue, (cap + 1) * sizeof(int))) != DG_OK) return r;
    if (h->Wf && (r = realloc_buf(h, h->Wf, (size_t)h->nv * h->N * cap * sizeof(float))) != DG_OK) return r;
    if (h->Wlo && (r = realloc_buf(h, h->Wlo, (size_t)h->nv * cap * sizeof(float))) != DG_OK) return r;
    h->cap_cells = cap;
  }
  if (nf > (int64_t)h->cap_faces) {
    const size_t cap = (size_t)grown(nf, INT32_MAX);
    MeshDev& m = h->md;
    if ((r = realloc_buf(h, m.fm, cap * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, m.fp, cap * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, m.finfo, cap)) != DG_OK) return r;
    if ((r = realloc_buf(h, h->F, (size_t)h->nv * h->ks->QF * cap * h->esize)) != DG_OK) return r;
    if (h->Gm && (r = realloc_buf(h, h->Gm, (size_t)h->nv * h->ks->QF * cap * sizeof(float))) != DG_OK) return r;
    if (h->Dm && (r = realloc_buf(h, h->Dm, (size_t)h->nv * cap * sizeof(float))) != DG_OK) return r;
    h->cap_faces = cap;
  }
  if (nn > (int64_t)h->cap_nodes) {
    const size_t cap = (size_t)grown(nn, h->bg.nbase);
    if ((r = realloc_buf(h, h->md.node_children, cap * nch * sizeof(int32_t))) != DG_OK) return r;
    h->cap_nodes = cap;
  }
  return DG_OK;
}

int ensure_scan_work(dg_handle* h, int64_t n) {
  const size_t need = scan_work_ints(n);
  if (need <= h->scan_work_cap) return DG_OK;
  const int r = realloc_buf(h, h->scan_work, need * sizeof(int32_t));
  if (r == DG_OK) h->scan_work_cap = need;
  return r;
}

// base maps and work arrays of the adaptation, on first use
int ensure_adapt(dg_handle* h) {
  if (h->adapt_crit) return DG_OK;
  if (h->nprob != 1) return fail(h, DG_ERR_UNSUPPORTED, "mesh adaptation needs a single problem");
  if (h->k < 1) return fail(h, DG_ERR_UNSUPPORTED, "mesh adaptation needs k >= 1 (the slope weights)");
  const int64_t nb = h->bg.nbase;
  if (nb * (1 << h->dim) * 3 * h->dim >= (int64_t)INT32_MAX)
    return fail(h, DG_ERR_UNSUPPORTED, "mesh adaptation: base grid too large for 32-bit face numbering");
  int r;
  for (int slot = 0; slot < 2; ++slot) {
    if ((r = realloc_buf(h, h->base_first[slot], (size_t)(nb + 1) * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, h->base_node[slot], (size_t)std::max<int64_t>(nb, 1) * sizeof(int32_t))) != DG_OK)
      return r;
  }
  h->cur = 0;
  DG_CUDA(h, cudaMemcpy(h->base_first[0], h->base_first_host.data(), (size_t)(nb + 1) * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
  DG_CUDA(h, cudaMemcpy(h->base_node[0], h->base_node_host.data(), (size_t)nb * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
  if ((r = realloc_buf(h, h->adapt_ref, (size_t)nb)) != DG_OK) return r;
  if ((r = realloc_buf(h, h->adapt_cnt, (size_t)nb * sizeof(int32_t))) != DG_OK) return r;
  if ((r = realloc_buf(h, h->adapt_info, sizeof(int32_t))) != DG_OK) return r;
  if ((r = ensure_scan_work(h, nb)) != DG_OK) return r;
  return realloc_buf(h, h->adapt_crit, (size_t)nb);
}

// prefix sum of the cells per base cell into the next slot, then the new
// sizes and the change count back to the host (synchronises the stream)
int finish_mark(dg_handle* h, int32_t* flags_host, int64_t* n_cells_new, int64_t* n_changed, cudaStream_t s) {
  const int nb = h->bg.nbase, nxt = 1 - h->cur;
  DG_CUDA(h, launch_scan(h->adapt_cnt, nb, h->base_first[nxt], h->scan_work, s));
  int32_t info[2] = {0, 0};
  DG_CUDA(h, cudaMemcpyAsync(&info[0], h->base_first[nxt] + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DG_CUDA(h, cudaMemcpyAsync(&info[1], h->adapt_info, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  std::vector<uint8_t> fl;
  if (flags_host) {
    fl.resize((size_t)nb);
    DG_CUDA(h, cudaMemcpyAsync(fl.data(), h->adapt_ref, (size_t)nb, cudaMemcpyDeviceToHost, s));
  }
  DG_CUDA(h, cudaStreamSynchronize(s));
  for (size_t b = 0; b < fl.size(); ++b) flags_host[b] = fl[b];
  h->next_cells = info[0];
  h->next_nodes = (info[0] - nb) / ((1 << h->dim) - 1);
  h->mark_pending = true;
  if (n_cells_new) *n_cells_new = info[0];
  if (n_changed) *n_changed = info[1];
  return DG_OK;
}

void drop_graphs(dg_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  for (auto& kv : h->pgraphs) {
    cudaGraphExecDestroy(kv.second.exec);
    for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
  }
  h->pgraphs.clear();
  for (auto g : h->graph_defs) cudaGraphDestroy(g);
  h->graph_defs.clear();
  for (auto& kv : h->plans) cudaFree(kv.second.first);  // (synchronises the device)
  h->plans.clear();
}

cudaError_t cell_launch(dg_handle* h, const void* args, cudaStream_t s) {
  if (h->use_tc) {
    h->tc_hook = 0;  // the hook (if armed) went with this launch's arguments
    return h->ks->cell_tc(args, s);
  }
  if (h->use_x2 && !h->accel) return h->ks->cell_x2(args, s);
  return h->use_direct && !h->accel ? h->ks->cell_direct(args, s) : h->ks->cell(args, s);
}

// face and cell kernels of one stage; DG_MIXED wraps the FP64 arguments.
// With delta registers (op given, h->delta) every scratch register holds the
// FP32 difference between its stage state and W.
template <typename real>
int stage_launch(dg_handle* h, const StageArgs<real>& a, cudaStream_t s, const Op* op = nullptr,
                 void* W = nullptr) {
  if constexpr (std::is_same<real, double>::value) {
    if (h->ms) {
      MixedArgs x;
      x.a = a;
      x.t = h->tab1d32;
      x.G = h->Gm;
      x.D = h->Dm;
      x.tcB = static_cast<const float*>(h->tcB);
      x.gamf = (float)h->gamma;
      x.g1f = x.gamf - 1.0f;
      if (op && h->delta) {
        auto freg = [&](int r) { return static_cast<float*>(h->regs[r - 1]); };
        x.delta = 1;
        x.a.U = static_cast<const double*>(W);
        x.R = op->in_reg == 0 ? nullptr : freg(op->in_reg);
        for (int r = 0; r < op->n_in; ++r) {
          if (op->in[r] == 0) continue;
          x.inR[x.n_inR] = freg(op->in[r]);
          x.Cf[x.n_inR] = (float)op->C[0][r];
          ++x.n_inR;
        }
        x.ckf = (float)op->ck[0];
        if (op->out[0] == 0) x.a.out[0] = static_cast<double*>(W);
        else x.outR = freg(op->out[0]);
        x.Wf = h->Wf;
        x.Wlo = h->Wlo;
        x.wf_mode = op->in_reg == 0 ? 1 : 2;
      }
      DG_CUDA(h, timed(h, DG_KERNEL_FACE, s, [&] { return h->ms->face(&x, s); }));
      if (h->use_tc) h->tc_hook = 0;  // the hook (if armed) went with this launch's arguments
      DG_CUDA(h, timed(h, DG_KERNEL_CELL, s,
                       [&] { return h->use_tc ? h->ms->cell_tc(&x, s) : h->ms->cell(&x, s); }));
      return DG_OK;
    }
  }
  if (h->use_fused && !h->use_tc && !h->use_direct && !h->use_x2 && !h->accel && h->nnodes == 0 && h->nprob == 1) {
    // faces computed inside the cell kernel's tiles: one launch per stage
    DG_CUDA(h, timed(h, DG_KERNEL_CELL, s, [&] { return h->ks->stage_fused(&a, s); }));
    return DG_OK;
  }
  DG_CUDA(h, timed(h, DG_KERNEL_FACE, s, [&] { return h->ks->face(&a, s); }));
  DG_CUDA(h, timed(h, DG_KERNEL_CELL, s, [&] { return cell_launch(h, &a, s); }));
  return DG_OK;
}

template <typename real>
StageArgs<real> stage_args(dg_handle* h, const Op& op, const void* U, void* W) {
  StageArgs<real> a;
  a.m = h->md;
  {
    const double* src = reinterpret_cast<const double*>(&h->tab1d64);
    real* dst = reinterpret_cast<real*>(&a.t1);
    for (size_t i = 0; i < sizeof(Tab1D<double>) / sizeof(double); ++i) dst[i] = (real)src[i];
  }
  for (int l = 0; l < 2; ++l) a.pre[l] = (real)(std::ldexp(1.0, 1 - h->dim) / std::ldexp(h->md.dx0, -l));
  a.pre_prob = h->nprob > 1 ? static_cast<const real*>(h->pre_prob) : nullptr;
  a.tcB = static_cast<const real*>(h->tcB);
  a.tc_hook = h->use_tc ? h->tc_hook : 0;
  a.status = h->status;
  a.tab = static_cast<const real*>(h->tab);
  a.U = static_cast<const real*>(U);
  a.F = static_cast<real*>(h->F);
  a.gamma = h->gamma;
  a.pdl = h->pdl;
  a.gam = (real)h->gamma;
  a.gm1 = (real)h->gamma - (real)1;
  auto reg = [&](int r) -> real* { return static_cast<real*>(r == 0 ? W : h->regs[r - 1]); };
  a.n_in = op.n_in;
  for (int r = 0; r < op.n_in; ++r) a.in[r] = reg(op.in[r]);
  a.n_out = op.n_out;
  for (int o = 0; o < op.n_out; ++o) {
    a.out[o] = reg(op.out[o]);
    a.ck[o] = (real)op.ck[o];
    for (int r = 0; r < MAX_IN; ++r) a.C[o][r] = (real)op.C[o][r];
  }
  a.dt = h->scal;
  a.accel = static_cast<const real*>(h->accel);
  a.cell_tile = h->cell_tile;
  a.face_tile = h->face_tile;
  a.dtab = h->dtab.empty() ? nullptr : h->dtab.data();
  return a;
}

template <typename real>
LimitArgs<real> limit_args(dg_handle* h, const void* src, void* dst) {
  LimitArgs<real> la;
  la.m = h->md;
  la.tab64 = h->tab64;
  la.tabr = static_cast<const real*>(h->tab);
  la.tab32 = h->tab32;
  la.Uin = static_cast<const real*>(src);
  la.Uout = static_cast<real*>(dst);
  la.gamma = h->gamma;
  la.pdl = h->pdl;
  la.limiter = h->opt.slope_limiter;
  la.beta = h->opt.beta;
  la.Mtilde = h->opt.Mtilde;
  la.positivity = h->opt.positivity;
  la.eps = h->opt.eps;
  la.fp32_slopes = h->ms != nullptr;  // DG_MIXED: FP32 slope-limiter arithmetic on the FP64 state
  la.counts = h->lim_counts;
  la.queue = h->lim_queue;
  la.queue_len = h->lim_queue + std::max(h->ncells, 1);
  la.status = h->status;
  return la;
}

template <typename real>
int run_limit(dg_handle* h, const void* src, void* dst, cudaStream_t s) {
  const LimitArgs<real> la = limit_args<real>(h, src, dst);
  DG_CUDA(h, timed(h, DG_KERNEL_LIMIT, s, [&] { return h->ks->limit(&la, s); }));
  return DG_OK;
}

template <typename real>
AuxArgs<real> aux_args(dg_handle* h) {
  AuxArgs<real> a;
  a.m = h->md;
  a.tab64 = h->tab64;
  a.partial = h->partial;
  a.gamma = h->gamma;
  a.pdl = h->pdl;
  a.volume = h->volume;
  for (int l = 0; l < 2; ++l) a.inv_dx[l] = 1.0 / std::ldexp(h->md.dx0, -l);
  a.inv_dx_prob = h->nprob > 1 ? h->inv_dx_prob : nullptr;
  a.dt_bits = h->dt_bits;
  a.status = h->status;
  a.accel = static_cast<const real*>(h->accel);
  return a;
}

double dt_factor(const dg_handle* h) {
  const double base = 1.0 / (2.0 * h->k + 1.0);
  if (!h->opt.positivity) return h->opt.cfl * base;
  std::vector<double> lx, lw;
  const int m = std::max(2, (h->k + 4) / 2);
  lobatto_rule(m, lx, lw);
  return h->opt.cfl * std::min(base, 0.5 * lw[0]);
}

template <typename real>
int compute_dt_impl(dg_handle* h, const void* W, double* copy, cudaStream_t s) {
  AuxArgs<real> a = aux_args<real>(h);
  a.W = static_cast<const real*>(W);
  const double fac = dt_factor(h);
  a.grav_factor = fac * std::sqrt(2.0 * h->gamma * (h->gamma - 1.0));
  if (h->ncells > 0) {
    // one launch: its last block finishes the timestep (dt_bits and dt_done
    // are zero between launches)
    a.dt_factor = fac;
    a.dt_out = h->scal;
    a.dt_copy = copy;
    a.dt_done = h->dt_done;
    DG_CUDA(h, timed(h, DG_KERNEL_DT, s, [&] { return h->ks->dt(&a, s); }));
    return DG_OK;
  }
  DG_CUDA(h, cudaMemsetAsync(h->dt_bits, 0, sizeof(unsigned long long) * h->nprob, s));
  DG_CUDA(h, timed(h, DG_KERNEL_OTHER, s,
                   [&] { return launch_dt_finalize(h->dt_bits, h->nprob, fac, h->scal, copy, s); }));
  return DG_OK;
}

// one step of the stage program on state W (register 0)
template <typename real>
int step_impl(dg_handle* h, const Program& P, void* W, cudaStream_t s) {
  for (const Op& op : P.ops) {
    void* U = op.in_reg == 0 ? W : h->regs[op.in_reg - 1];
    StageArgs<real> a = stage_args<real>(h, op, U, W);
    const int rs = stage_launch<real>(h, a, s, &op, W);
    if (rs != DG_OK) return rs;
    if (op.lim_src >= 0) {
      void* src = op.lim_src == 0 ? W : h->regs[op.lim_src - 1];
      void* dst = op.lim_dst == 0 ? W : h->regs[op.lim_dst - 1];
      const int r = run_limit<real>(h, src, dst, s);
      if (r != DG_OK) return r;
    }
  }
  return DG_OK;
}

template <typename real>
int rk_step_any(dg_handle* h, void* W, double dt, double* dt_used, cudaStream_t s) {
  if (dt > 0.0) {
    DG_CUDA(h, timed(h, DG_KERNEL_OTHER, s, [&] { return launch_set_scalar(h->scal, h->nprob, dt, s); }));
    if (dt_used)
      DG_CUDA(h, timed(h, DG_KERNEL_OTHER, s,
                       [&] { return launch_set_scalar(dt_used, h->nprob, dt, s); }));
  } else {
    const int r = compute_dt_impl<real>(h, W, dt_used, s);
    if (r != DG_OK) return r;
  }
  return step_impl<real>(h, h->prog_step, W, s);
}

// dg_advance with the persistent whole-step kernel: the handle supports it
// (2D, an FP64 or FP32 state with the CUDA-core stage kernels, no gravity
// source, at most PERSIST_MAX_OPS stages)
bool persist_supported(const dg_handle* h) {
  return h->ks->persist && !h->ms && !h->use_tc && !h->use_direct && !h->use_x2 && !h->accel && h->ncells > 0 &&
         (int)h->prog_step.ops.size() <= PERSIST_MAX_OPS;
}

// the plan of one step on state W (dt history at hist, or none), built once
// per (W, hist) and kept in device memory until the graphs are dropped
template <typename real>
int persist_plan(dg_handle* h, void* W, double* hist, void** plan_dev, int* max_blocks) {
  const auto key = std::make_pair(W, static_cast<void*>(hist));
  auto it = h->plans.find(key);
  if (it == h->plans.end()) {
    std::unique_ptr<PersistPlan<real>> P(new PersistPlan<real>());
    const Program& prog = h->prog_step;
    P->n_ops = (int)prog.ops.size();
    for (int i = 0; i < P->n_ops; ++i) {
      const Op& op = prog.ops[i];
      void* U = op.in_reg == 0 ? W : h->regs[op.in_reg - 1];
      P->op[i].st = stage_args<real>(h, op, U, W);
      if (op.lim_src >= 0) {
        void* src = op.lim_src == 0 ? W : h->regs[op.lim_src - 1];
        void* dst = op.lim_dst == 0 ? W : h->regs[op.lim_dst - 1];
        P->op[i].lim = 1;
        P->op[i].la = limit_args<real>(h, src, dst);
      }
    }
    AuxArgs<real> a = aux_args<real>(h);
    a.W = static_cast<const real*>(W);
    const double fac = dt_factor(h);
    a.grav_factor = fac * std::sqrt(2.0 * h->gamma * (h->gamma - 1.0));
    a.dt_factor = fac;
    a.dt_out = h->scal;
    a.dt_copy = hist;
    a.dt_done = h->dt_done;
    P->dt = a;
    const int nc = h->ncells, nf = std::max(h->nfaces, 0);
    P->face_blocks = (nf + 31) / 32;
    P->cell_blocks = (nc + 31) / 32;
    P->lim_blocks = (nc + 127) / 128;
    P->pos_blocks = std::min((nc + 127) / 128, 608);
    P->dt_blocks = (nc + 127) / 128;
    const int mb = std::max({P->face_blocks, P->cell_blocks, P->lim_blocks, P->pos_blocks, P->dt_blocks});
    void* d = nullptr;
    DG_CUDA(h, cudaMalloc(&d, sizeof(PersistPlan<real>)));
    const cudaError_t e = cudaMemcpy(d, P.get(), sizeof(PersistPlan<real>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(h, e, "cudaMemcpy step plan");
    }
    it = h->plans.emplace(key, std::make_pair(d, mb)).first;
  }
  *plan_dev = it->second.first;
  *max_blocks = it->second.second;
  return DG_OK;
}

template <typename real>
int advance_persistent(dg_handle* h, void* W, int n_steps, double* hist, cudaStream_t s) {
  void* plan = nullptr;
  int mb = 0;
  const int r = persist_plan<real>(h, W, hist, &plan, &mb);
  if (r != DG_OK) return r;
  DG_CUDA(h, cudaMemsetAsync(h->bar, 0, 4 * sizeof(unsigned), s));
  DG_CUDA(h, timed(h, DG_KERNEL_OTHER, s, [&] { return h->ks->persist(plan, mb, n_steps, h->bar, h->status, s); }));
  return DG_OK;
}

template <typename real>
int combine_list(dg_handle* h, void* out, const std::vector<std::pair<double, const void*>>& terms,
                 cudaStream_t s) {
  CombineArgs<real> c;
  c.out = static_cast<real*>(out);
  c.n = (size_t)h->nv * h->N * h->ncells;
  for (const auto& t : terms) {
    if (t.first == 0.0) continue;
    if (c.n_terms >= MAX_COMBINE) return fail(h, DG_ERR_ARG, "internal: too many combine terms");
    c.c[c.n_terms] = (real)t.first;
    c.x[c.n_terms] = static_cast<const real*>(t.second);
    ++c.n_terms;
  }
  DG_CUDA(h, timed(h, DG_KERNEL_OTHER, s, [&] { return h->ks->combine(&c, s); }));
  return DG_OK;
}

// dW/dt(U) -> out (no stage combination)
template <typename real>
int rhs_into(dg_handle* h, const void* U, void* out, cudaStream_t s) {
  Op op;
  op.n_in = 0;
  op.n_out = 1;
  op.ck[0] = 1.0;
  StageArgs<real> a = stage_args<real>(h, op, U, nullptr);
  a.out[0] = static_cast<real*>(out);
  a.dt = nullptr;
  return stage_launch<real>(h, a, s);
}

// acc = J(U)^T G, J the Jacobian of dW/dt
template <typename real>
int adjoint_rhs_into(dg_handle* h, const void* U, const void* G, void* acc, cudaStream_t s) {
  AdjointArgs<real> a;
  a.m = h->md;
  {
    const double* src = reinterpret_cast<const double*>(&h->tab1d64);
    real* dst = reinterpret_cast<real*>(&a.t1);
    for (size_t i = 0; i < sizeof(Tab1D<double>) / sizeof(double); ++i) dst[i] = (real)src[i];
  }
  for (int l = 0; l < 2; ++l) a.pre[l] = (real)(std::ldexp(1.0, 1 - h->dim) / std::ldexp(h->md.dx0, -l));
  a.pre_prob = h->nprob > 1 ? static_cast<const real*>(h->pre_prob) : nullptr;
  a.U = static_cast<const real*>(U);
  a.G = static_cast<const real*>(G);
  a.FG = static_cast<real*>(h->FG);
  a.acc = static_cast<real*>(acc);
  a.gamma = h->gamma;
  a.scale = 1.0;
  DG_CUDA(h, timed(h, DG_KERNEL_ADJOINT, s, [&] { return h->ks->adj_face(&a, s); }));
  DG_CUDA(h, timed(h, DG_KERNEL_ADJOINT, s, [&] { return h->ks->adj_cell(&a, s); }));
  return DG_OK;
}

// Adjoint of one step in Butcher form with frozen dt:
//   k_i = L(U_i), U_i = w + dt sum_{j<i} a_ij k_j, w' = w + dt sum_i b_i k_i
//   kbar_i = dt (b_i lam + sum_{m>i} a_mi Ubar_m),  Ubar_i = J(U_i)^T kbar_i,
//   lam_n = lam + sum_i Ubar_i.
template <typename real>
int adjoint_step_impl(dg_handle* h, const void* Wn, double dt, const void* lam1, void* lam0,
                      cudaStream_t s) {
  const Tab tb = butcher(h->opt.rk_order);
  const int S = tb.s;
  const size_t bytes = (size_t)h->nv * h->N * h->ncells * h->esize;
  while ((int)h->adj.size() < 2 * S) {
    void* p = nullptr;
    const int r = dalloc(h, bytes, &p);
    if (r != DG_OK) return r;
    h->adj.push_back(p);
  }
  if (!h->FG) {
    const int r = dalloc(h, (size_t)2 * h->nv * h->ks->QF * std::max(h->nfaces, 1) * h->esize, &h->FG);
    if (r != DG_OK) return r;
  }
  auto U = [&](int i) -> void* { return i == 0 ? const_cast<void*>(Wn) : h->adj[i - 1]; };
  auto Kb = [&](int i) -> void* { return h->adj[S - 1 + i]; };
  void* kbar = h->adj[2 * S - 1];
  int r;
  // stage states from the checkpoint
  for (int i = 0; i < S; ++i) {
    if ((r = rhs_into<real>(h, U(i), Kb(i), s)) != DG_OK) return r;
    if (i + 1 < S) {
      std::vector<std::pair<double, const void*>> t{{1.0, Wn}};
      for (int j = 0; j <= i; ++j) t.push_back({dt * tb.A[(i + 1) * S + j], Kb(j)});
      if ((r = combine_list<real>(h, U(i + 1), t, s)) != DG_OK) return r;
    }
  }
  // reverse sweep; Ubar_i replaces k_i in Kb(i)
  for (int i = S - 1; i >= 0; --i) {
    std::vector<std::pair<double, const void*>> t{{dt * tb.b[i], lam1}};
    for (int m = i + 1; m < S; ++m) t.push_back({dt * tb.A[m * S + i], Kb(m)});
    if ((r = combine_list<real>(h, kbar, t, s)) != DG_OK) return r;
    if ((r = adjoint_rhs_into<real>(h, U(i), kbar, Kb(i), s)) != DG_OK) return r;
  }
  std::vector<std::pair<double, const void*>> t{{1.0, lam1}};
  for (int i = 0; i < S; ++i) t.push_back({1.0, Kb(i)});
  return combine_list<real>(h, lam0, t, s);
}

// Tile autotuner: times RK steps of a free-stream state on the handle's own
// mesh for every feasible tile of the face kernel (cell tile fixed), then of
// the cell kernel (and, for FP32 2D handles, the one-thread-per-cell kernel),
// keeping the fastest of each.
template <typename real>
int autotune_tiles(dg_handle* h, cudaStream_t s) {
  const size_t n = (size_t)h->nv * h->N * h->ncells;
  if (n == 0) return DG_OK;
  void* U = nullptr;
  int r;
  if (cudaMalloc(&U, n * h->esize) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, DG_ERR_OOM, "autotune: out of device memory");
  }
  struct Free {
    void* a;
    ~Free() { cudaFree(a); }
  } guard{U};
  // rho = 1, m = 0, E = 2.5 (p = 1 at gamma = 1.4): weight 0 of each variable
  DG_CUDA(h, launch_fill(U, n, 0.0, (int)h->esize, s));
  const size_t row = (size_t)h->N * h->ncells;
  DG_CUDA(h, launch_fill(U, h->ncells, 1.0, (int)h->esize, s));
  DG_CUDA(h, launch_fill(static_cast<char*>(U) + (h->nv - 1) * row * h->esize, h->ncells,
                         1.0 / (h->gamma - 1.0), (int)h->esize, s));
  // the two timing events, destroyed on every return path
  struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  DG_CUDA(h, cudaEventCreate(&ev.e[0]));
  DG_CUDA(h, cudaEventCreate(&ev.e[1]));
  cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
  // a full step of the handle's own stage program (fixed dt, so no timestep
  // reduction): the epilogues and registers the step really uses
  auto time_rhs = [&](float& best) -> int {
    best = 3.4e38f;
    for (int trial = 0; trial < 3; ++trial) {
      const int rr = rk_step_any<real>(h, U, 1e-9, nullptr, s);
      if (rr != DG_OK) return rr;
      DG_CUDA(h, cudaEventRecord(e0, s));
      for (int rep = 0; rep < 3; ++rep) {
        const int r2 = rk_step_any<real>(h, U, 1e-9, nullptr, s);
        if (r2 != DG_OK) return r2;
      }
      DG_CUDA(h, cudaEventRecord(e1, s));
      DG_CUDA(h, cudaEventSynchronize(e1));
      float ms = 0.0f;
      DG_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, ms);
    }
    return DG_OK;
  };
  const int cmax = h->ms ? h->ms->cell_tile_max : h->ks->cell_tile_max;
  const int fmax = h->ms ? h->ms->face_tile_max : h->ks->face_tile_max;
  const int cdef = h->ms ? h->ms->cell_tile : h->ks->cell_tile;
  const int fdef = h->ms ? h->ms->face_tile : h->ks->face_tile;
  // a candidate replaces the default only when it is faster by more than the
  // trials' noise (3%)
  constexpr float kMargin = 0.97f;
  h->cell_tile = cdef;
  int best_f = fdef;
  float best_t = 3.4e38f, def_t = 3.4e38f;
  for (int fb = 16; fb <= fmax; fb *= 2) {
    h->face_tile = fb;
    float t;
    if ((r = time_rhs(t)) != DG_OK) return r;
    if (fb == fdef) def_t = t;
    if (t < best_t) { best_t = t; best_f = fb; }
  }
  if (best_f != fdef && !(best_t < kMargin * def_t)) best_f = fdef;
  h->face_tile = best_f;
  if (!h->use_tc) {
    int best_c = cdef;
    bool best_direct = false;
    best_t = 3.4e38f;
    def_t = 3.4e38f;
    for (int tc = 16; tc <= cmax; tc *= 2) {
      h->cell_tile = tc;
      float t;
      if ((r = time_rhs(t)) != DG_OK) return r;
      if (tc == cdef) def_t = t;
      if (t < best_t) { best_t = t; best_c = tc; }
    }
    if (!h->dtab.empty()) {  // one thread per cell
      h->use_direct = true;
      float t;
      if ((r = time_rhs(t)) != DG_OK) return r;
      if (t < best_t) { best_t = t; best_direct = true; }
      h->use_direct = false;
    }
    bool best_x2 = false;
    if (h->ks->cell_x2 && !h->ms) {  // two variables per thread, packed FP32 pairs
      h->use_x2 = true;
      float t;
      if ((r = time_rhs(t)) != DG_OK) return r;
      if (t < best_t) { best_t = t; best_x2 = true; best_direct = false; }
      h->use_x2 = false;
    }
    if ((best_direct || best_x2 || best_c != cdef) && !(best_t < kMargin * def_t)) {
      best_c = cdef;
      best_direct = false;
      best_x2 = false;
    }
    h->cell_tile = best_c;
    h->use_direct = best_direct;
    h->use_x2 = best_x2;
  }
  DG_CUDA(h, cudaStreamSynchronize(s));
  return DG_OK;
}

int rk_step_dispatch(dg_handle* h, void* W, double dt, double* dt_used, cudaStream_t s) {
  return h->prec == DG_FP64 ? rk_step_any<double>(h, W, dt, dt_used, s)
                            : rk_step_any<float>(h, W, dt, dt_used, s);
}

bool check_handle(const dg_handle* h) { return h != nullptr && h->ks != nullptr; }

// a handle whose gravity field was dropped by a regrid must get a new one
int check_gravity(dg_handle* h, const char* who) {
  if (!h->accel_stale) return DG_OK;
  return fail(h, DG_ERR_ARG, std::string(who) + ": the gravity field was sampled on the mesh before the "
                                                "last dg_regrid; set it again (dg_set_gravity)");
}

}  // namespace

// ===========================================================================
extern "C" {

int dg_default_options(dg_options* opt) {
  if (!opt) return DG_ERR_ARG;
  opt->rk_order = 3;
  opt->cfl = 0.2;
  opt->slope_limiter = DG_LIMITER_NONE;
  opt->beta = 1.0;
  opt->Mtilde = 0.5;
  opt->positivity = 0;
  opt->eps = 1e-10;
  opt->precision = DG_FP64;
  opt->autotune = 0;
  opt->basis = DG_BASIS_TOTAL;
  return DG_OK;
}

const char* dg_last_error(const dg_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

// the tensor-product basis has the stage, timestep, projection and
// diagnostic kernels only
static int tensor_unsupported(dg_handle* h, const char* what) {
  if (h->ks->basis == 0) return DG_OK;
  return fail(h, DG_ERR_UNSUPPORTED, std::string(what) + ": not built for the tensor-product basis");
}

static int create_impl(const dg_mesh_desc* mesh, int nprob, int k, double gamma,
                       const dg_options* opt, dg_handle** out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "dg_create: out is NULL");
  *out = nullptr;
  if (!mesh) return fail(nullptr, DG_ERR_ARG, "dg_create: mesh is NULL");
  if (nprob < 1) return fail(nullptr, DG_ERR_ARG, "dg_create_batch: n_problems must be >= 1");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, DG_ERR_ARG, "dg_create: dim must be 2 or 3");
  if (!(gamma > 1.0)) return fail(nullptr, DG_ERR_ARG, "dg_create: gamma must exceed 1");
  dg_options o;
  dg_default_options(&o);
  if (opt) o = *opt;
  if (o.rk_order < 1 || o.rk_order > 4) return fail(nullptr, DG_ERR_ARG, "dg_create: rk_order must be 1..4");
  if (o.slope_limiter < 0 || o.slope_limiter > 2) return fail(nullptr, DG_ERR_ARG, "dg_create: bad slope_limiter");
  if (o.precision != DG_FP64 && o.precision != DG_FP32 && o.precision != DG_FP32_TC &&
      o.precision != DG_MIXED && o.precision != DG_MIXED_TC)
    return fail(nullptr, DG_ERR_ARG, "dg_create: bad precision");
  const bool use_tc = o.precision == DG_FP32_TC || o.precision == DG_MIXED_TC;
  const bool mixed = o.precision == DG_MIXED || o.precision == DG_MIXED_TC;
  if (use_tc) o.precision = DG_FP32;
  if (mixed) o.precision = DG_FP64;  // FP64 state; FP32 stage kernels below
  if (!(o.cfl > 0.0)) return fail(nullptr, DG_ERR_ARG, "dg_create: cfl must be positive");
  if (o.basis != DG_BASIS_TOTAL && o.basis != DG_BASIS_TENSOR) return fail(nullptr, DG_ERR_ARG, "dg_create: bad basis");
  if (o.basis == DG_BASIS_TENSOR && k > 0 &&
      (mesh->dim != 2 || use_tc || mixed || o.slope_limiter != DG_LIMITER_NONE || o.positivity))
    return fail(nullptr, DG_ERR_UNSUPPORTED,
                "dg_create: the tensor-product basis needs dim 2, an FP64 or FP32 state and no limiter");
  const KernelSet* ks = kernel_set(o.precision, mesh->dim, k, o.basis);
  if (!ks) return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_create: (dim, k, precision, basis) not compiled");
  auto* h = new dg_handle();
  h->dim = mesh->dim;
  h->k = k;
  h->prec = o.precision;
  h->gamma = gamma;
  h->opt = o;
  h->ks = ks;
  h->use_tc = use_tc;
  h->nv = ks->NV;
  h->N = ks->N;
  h->esize = o.precision == DG_FP64 ? 8 : 4;
  auto bail = [&](int code) {
    g_create_error = h->err;
    dg_destroy(h);
    return code;
  };
  int r = nprob == 1 ? build_mesh(h, mesh) : build_batch(h, mesh, nprob);
  if (r != DG_OK) return bail(r);
  // tables
  std::vector<double> gx, gw, g3x, g3w, lx, lw, T;
  gauss_rule(k + 1, gx, gw);
  gauss_rule(k + 3, g3x, g3w);
  lobatto_rule(std::max(2, (k + 4) / 2), lx, lw);
  ks->fill_tables(T, gx, gw, g3x, g3w, lx);
  std::memcpy(&h->tab1d64, &T[T.size() - sizeof(Tab1D<double>) / sizeof(double)], sizeof(Tab1D<double>));
  void* p = nullptr;
  if ((r = dalloc(h, T.size() * sizeof(double), &p)) != DG_OK) return bail(r);
  h->tab64 = static_cast<double*>(p);
  if (cudaMemcpy(h->tab64, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "cudaMemcpy tables"));
  {
    std::vector<float> Tf(T.begin(), T.end());
    if ((r = dalloc(h, Tf.size() * sizeof(float), &p)) != DG_OK) return bail(r);
    h->tab32 = static_cast<float*>(p);
    if (cudaMemcpy(p, Tf.data(), Tf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(cuda_fail(h, cudaGetLastError(), "cudaMemcpy tables"));
  }
  h->tab = h->prec == DG_FP64 ? static_cast<void*>(h->tab64) : static_cast<void*>(h->tab32);
  // mesh tables
  if ((r = upload(h, h->level, &h->md.level)) != DG_OK) return bail(r);
  if ((r = upload(h, h->coord, &h->md.coord)) != DG_OK) return bail(r);
  if ((r = upload(h, h->nbr, &h->md.nbr)) != DG_OK) return bail(r);
  if ((r = upload(h, h->fm, &h->md.fm)) != DG_OK) return bail(r);
  if ((r = upload(h, h->fp, &h->md.fp)) != DG_OK) return bail(r);
  if ((r = upload(h, h->finfo, &h->md.finfo)) != DG_OK) return bail(r);
  if ((r = upload(h, h->sface, &h->md.sface)) != DG_OK) return bail(r);
  if ((r = upload(h, h->scoarse, &h->md.scoarse)) != DG_OK) return bail(r);
  if ((r = upload(h, h->node_children, &h->md.node_children)) != DG_OK) return bail(r);
  if (h->nprob > 1) {
    if ((r = upload(h, h->prob, &h->md.prob)) != DG_OK) return bail(r);
    if ((r = upload(h, h->dx_prob, &h->md.dx_prob)) != DG_OK) return bail(r);
    if ((r = upload(h, h->lo_prob, &h->md.lo_prob)) != DG_OK) return bail(r);
    std::vector<double> pre(h->nprob), inv(h->nprob);
    for (int p = 0; p < h->nprob; ++p) {
      pre[p] = std::ldexp(1.0, 1 - h->dim) / h->dx_prob[p];
      inv[p] = 1.0 / h->dx_prob[p];
    }
    const double* dinv = nullptr;
    if ((r = upload(h, inv, &dinv)) != DG_OK) return bail(r);
    h->inv_dx_prob = const_cast<double*>(dinv);
    if (h->prec == DG_FP64) {
      const double* dp = nullptr;
      if ((r = upload(h, pre, &dp)) != DG_OK) return bail(r);
      h->pre_prob = const_cast<double*>(dp);
    } else {
      std::vector<float> pref(pre.begin(), pre.end());
      const float* dp = nullptr;
      if ((r = upload(h, pref, &dp)) != DG_OK) return bail(r);
      h->pre_prob = const_cast<float*>(dp);
    }
  }
  // stage programs and scratch
  std::string perr;
  const bool limited = (o.slope_limiter != DG_LIMITER_NONE && k > 0) || (o.positivity && k > 0);
  if (!build_program(o.rk_order, limited, h->prog_step, perr)) return bail(fail(h, DG_ERR_ARG, perr));
  if (!build_program(o.rk_order, false, h->prog_free, perr)) return bail(fail(h, DG_ERR_ARG, perr));
  const size_t state_bytes = (size_t)h->nv * h->N * h->ncells * h->esize;
  const int nregs = std::max(h->prog_step.n_phys, h->prog_free.n_phys) + 1;
  for (int i = 0; i < nregs; ++i) {
    if ((r = dalloc(h, state_bytes, &p)) != DG_OK) return bail(r);
    h->regs.push_back(p);
  }
  if ((r = dalloc(h, (size_t)h->nv * ks->QF * std::max(h->nfaces, 1) * h->esize, &h->F)) != DG_OK)
    return bail(r);
  if ((r = dalloc(h, (size_t)h->nprob * sizeof(double), &p)) != DG_OK) return bail(r);
  h->scal = static_cast<double*>(p);
  if ((r = dalloc(h, (size_t)h->nprob * sizeof(unsigned long long), &p)) != DG_OK) return bail(r);
  h->dt_bits = static_cast<unsigned long long*>(p);
  if (cudaMemset(h->dt_bits, 0, (size_t)h->nprob * sizeof(unsigned long long)) != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "cudaMemset"));
  if ((r = dalloc(h, sizeof(unsigned int), &p)) != DG_OK) return bail(r);
  h->dt_done = static_cast<unsigned int*>(p);
  if (cudaMemset(h->dt_done, 0, sizeof(unsigned int)) != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "cudaMemset"));
  const int nblk = (h->ncells + 255) / 256 + 1;
  if ((r = dalloc(h, (size_t)nblk * 8 * sizeof(double), &p)) != DG_OK) return bail(r);
  h->partial = static_cast<double*>(p);
  if ((r = dalloc(h, sizeof(int), &p)) != DG_OK) return bail(r);
  h->status = static_cast<int*>(p);
  if ((r = dalloc(h, 3 * sizeof(unsigned long long), &p)) != DG_OK) return bail(r);
  h->lim_counts = static_cast<unsigned long long*>(p);
  if ((r = dalloc(h, ((size_t)std::max(h->ncells, 1) + 1) * sizeof(int), &p)) != DG_OK) return bail(r);
  h->lim_queue = static_cast<int*>(p);
  if (cudaMemset(h->lim_counts, 0, 3 * sizeof(unsigned long long)) != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "cudaMemset"));
  if (cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "cudaMemset"));
  if (ks->prepare() != cudaSuccess) return bail(cuda_fail(h, cudaGetLastError(), "kernel attributes"));
  if (mixed) {
    h->ms = mixed_set(h->dim, k);
    if (!h->ms) return bail(fail(h, DG_ERR_UNSUPPORTED, "dg_create: DG_MIXED not compiled for (dim, k)"));
    if (h->ms->prepare() != cudaSuccess)
      return bail(cuda_fail(h, cudaGetLastError(), "kernel attributes"));
    const double* src = reinterpret_cast<const double*>(&h->tab1d64);
    float* dst = reinterpret_cast<float*>(&h->tab1d32);
    for (size_t i = 0; i < sizeof(Tab1D<double>) / sizeof(double); ++i) dst[i] = (float)src[i];
    const size_t nf = (size_t)std::max(h->nfaces, 1);
    // delta registers: unlimited program whose stage states are affine
    // combinations (coefficients summing to one) of W and earlier stage states
    h->delta = !limited;
    for (const Op& op : h->prog_step.ops) {
      double sum = 0.0;
      for (int r = 0; r < op.n_in; ++r) sum += op.C[0][r];
      if (op.n_out != 1 || op.lim_src >= 0 || std::fabs(sum - 1.0) > 1e-12) h->delta = false;
    }
    if (h->delta) {
      if ((r = dalloc(h, (size_t)h->nv * h->N * std::max(h->ncells, 1) * sizeof(float), &p)) != DG_OK)
        return bail(r);
      h->Wf = static_cast<float*>(p);
      if ((r = dalloc(h, (size_t)h->nv * std::max(h->ncells, 1) * sizeof(float), &p)) != DG_OK) return bail(r);
      h->Wlo = static_cast<float*>(p);
    }
    if ((r = dalloc(h, (size_t)h->nv * ks->QF * nf * sizeof(float), &p)) != DG_OK) return bail(r);
    h->Gm = static_cast<float*>(p);
    if ((r = dalloc(h, (size_t)h->nv * nf * sizeof(float), &p)) != DG_OK) return bail(r);
    h->Dm = static_cast<float*>(p);
  }
  if (!h->ms && !use_tc && ks->fill_direct) ks->fill_direct(T, h->dtab);
  if (h->use_tc) {
    auto cell_tc = h->ms ? h->ms->cell_tc : ks->cell_tc;
    auto prepare_tc = h->ms ? h->ms->prepare_tc : ks->prepare_tc;
    auto fill_tc = h->ms ? h->ms->fill_tc : ks->fill_tc;
    if (!cell_tc || h->nnodes > 0)
      return bail(fail(h, DG_ERR_UNSUPPORTED,
                       "dg_create: tensor-core precisions need a uniform 2D mesh and k = 1..3"));
    if (prepare_tc() != cudaSuccess)
      return bail(cuda_fail(h, cudaGetLastError(), "kernel attributes"));
    std::vector<float> B;
    fill_tc(T, B);
    if ((r = dalloc(h, B.size() * sizeof(float), &p)) != DG_OK) return bail(r);
    h->tcB = p;
    if (cudaMemcpy(p, B.data(), B.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(cuda_fail(h, cudaGetLastError(), "cudaMemcpy tensor-core tables"));
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "cudaStreamCreate"));
  h->cell_tile = h->ms ? h->ms->cell_tile : ks->cell_tile;
  h->face_tile = h->ms ? h->ms->face_tile : ks->face_tile;
  h->cap_cells = (size_t)h->ncells;
  h->cap_faces = (size_t)std::max(h->nfaces, 1);
  h->cap_nodes = (size_t)h->nnodes;
  if (o.autotune) {
    r = h->prec == DG_FP64 ? autotune_tiles<double>(h, h->cap_stream)
                           : autotune_tiles<float>(h, h->cap_stream);
    if (r != DG_OK) return bail(r);
  }
  // the persistent whole-step kernel, an alternative for dg_advance
  // (dg_set_advance_mode); the graph stays the default: it measured faster
  // on every mesh size tried, down to 32^2 cells
  if (ks->persist && ks->prepare_persist) {
    if ((r = dalloc(h, 4 * sizeof(unsigned), &p)) != DG_OK) return bail(r);
    h->bar = static_cast<unsigned*>(p);
    if (ks->prepare_persist() != cudaSuccess) return bail(cuda_fail(h, cudaGetLastError(), "kernel attributes"));
  }
  if (ks->prepare_fused && !h->ms && !h->use_tc && ks->prepare_fused() != cudaSuccess)
    return bail(cuda_fail(h, cudaGetLastError(), "kernel attributes"));
  *out = h;
  return DG_OK;
}

int dg_create(const dg_mesh_desc* mesh, int k, double gamma, const dg_options* opt,
              dg_handle** out) {
  return create_impl(mesh, 1, k, gamma, opt, out);
}

int dg_create_batch(const dg_mesh_desc* meshes, const double* gamma, int n_problems, int k,
                    const dg_options* opt, dg_handle** out) {
  if (!meshes || !gamma || n_problems < 1) {
    if (out) *out = nullptr;
    return fail(nullptr, DG_ERR_ARG, "dg_create_batch: bad arguments");
  }
  for (int p = 1; p < n_problems; ++p)
    if (gamma[p] != gamma[0]) {
      if (out) *out = nullptr;
      return fail(nullptr, DG_ERR_UNSUPPORTED, "dg_create_batch: problems must share gamma");
    }
  return create_impl(meshes, n_problems, k, gamma[0], opt, out);
}

int dg_destroy(dg_handle* h) {
  if (!h) return DG_OK;
  cudaDeviceSynchronize();
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : h->pgraphs) {
    cudaGraphExecDestroy(kv.second.exec);
    for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
  }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (auto g : h->graph_defs) cudaGraphDestroy(g);
  for (auto& kv : h->plans) cudaFree(kv.second.first);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
  return DG_OK;
}

int dg_sizes(const dg_handle* h, int64_t* n_cells, int* n_basis, int* n_vars, int* n_qpoints,
             int* n_l1points, int* n_nodes) {
  if (!check_handle(h)) return DG_ERR_ARG;
  if (n_cells) *n_cells = h->ncells;
  if (n_basis) *n_basis = h->N;
  if (n_vars) *n_vars = h->nv;
  if (n_qpoints) *n_qpoints = h->ks->Q;
  if (n_l1points) *n_l1points = h->ks->Q1;
  if (n_nodes) *n_nodes = h->nnodes;
  return DG_OK;
}

static int points_impl(const dg_handle* hc, double* xyz, int l1, void* stream) {
  dg_handle* h = const_cast<dg_handle*>(hc);
  if (!check_handle(h) || !xyz) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->prec == DG_FP64) {
    AuxArgs<double> a = aux_args<double>(h);
    a.out = xyz;
    DG_CUDA(h, h->ks->points(&a, l1, s));
  } else {
    AuxArgs<float> a = aux_args<float>(h);
    a.out = xyz;
    DG_CUDA(h, h->ks->points(&a, l1, s));
  }
  return DG_OK;
}

int dg_quad_points(const dg_handle* h, double* xyz_dev, void* stream) {
  return points_impl(h, xyz_dev, 0, stream);
}
int dg_l1_points(const dg_handle* h, double* xyz_dev, void* stream) {
  return points_impl(h, xyz_dev, 1, stream);
}

int dg_project(dg_handle* h, const double* u_dev, void* W_dev, void* stream) {
  if (!check_handle(h) || !u_dev || !W_dev) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->prec == DG_FP64) {
    AuxArgs<double> a = aux_args<double>(h);
    a.u = u_dev;
    a.Wout = static_cast<double*>(W_dev);
    DG_CUDA(h, h->ks->project(&a, s));
  } else {
    AuxArgs<float> a = aux_args<float>(h);
    a.u = u_dev;
    a.Wout = static_cast<float*>(W_dev);
    DG_CUDA(h, h->ks->project(&a, s));
  }
  return DG_OK;
}

int dg_limiter_counts(dg_handle* h, int64_t* counts_dev, int reset, void* stream) {
  if (!check_handle(h) || !counts_dev) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DG_CUDA(h, cudaMemcpyAsync(counts_dev, h->lim_counts, 3 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToDevice, s));
  if (reset) DG_CUDA(h, cudaMemsetAsync(h->lim_counts, 0, 3 * sizeof(unsigned long long), s));
  return DG_OK;
}

int dg_set_tiles(dg_handle* h, int cell_tile, int face_tile) {
  if (!check_handle(h)) return DG_ERR_ARG;
  const int cmax = h->ms ? h->ms->cell_tile_max : h->ks->cell_tile_max;
  const int fmax = h->ms ? h->ms->face_tile_max : h->ks->face_tile_max;
  if (face_tile == 0) {
    if (!h->ks->stage_fused || h->ms || h->use_tc || h->nnodes > 0 || h->nprob != 1 || cell_tile == 1 ||
        cell_tile == 2)
      return fail(h, DG_ERR_UNSUPPORTED,
                  "dg_set_tiles: the fused face + cell kernel needs a single 2D uniform mesh with an FP64 or "
                  "FP32 state and the CUDA-core cell kernel");
  } else {
    if (face_tile != 16 && face_tile != 32 && face_tile != 64) return fail(h, DG_ERR_ARG, "dg_set_tiles: face tile");
    if (face_tile > fmax) return fail(h, DG_ERR_UNSUPPORTED, "dg_set_tiles: face tile too large for (dim, k)");
  }
  if (cell_tile == 1) {
    if (h->use_tc || h->dtab.empty())
      return fail(h, DG_ERR_UNSUPPORTED, "dg_set_tiles: one thread per cell needs an FP32 2D handle");
  } else if (cell_tile == 2) {
    if (h->use_tc || h->ms || !h->ks->cell_x2)
      return fail(h, DG_ERR_UNSUPPORTED, "dg_set_tiles: the packed-pair cell kernel needs an FP32 2D handle");
  } else {
    if (cell_tile != 16 && cell_tile != 32 && cell_tile != 64) return fail(h, DG_ERR_ARG, "dg_set_tiles: cell tile");
    if (cell_tile > cmax) return fail(h, DG_ERR_UNSUPPORTED, "dg_set_tiles: cell tile too large for (dim, k)");
  }
  std::lock_guard<std::mutex> lock(h->mu);
  h->use_fused = face_tile == 0;
  if (face_tile != 0) h->face_tile = face_tile;
  h->use_direct = cell_tile == 1;
  h->use_x2 = cell_tile == 2;
  if (cell_tile != 1 && cell_tile != 2) h->cell_tile = cell_tile;
  // cached step graphs hold the old launch configuration: record them anew
  drop_graphs(h);
  return DG_OK;
}

int dg_tiles(const dg_handle* h, int* cell_tile, int* face_tile) {
  if (!check_handle(h) || !cell_tile || !face_tile) return DG_ERR_ARG;
  *cell_tile = h->use_tc ? 128 : (h->use_direct ? 1 : (h->use_x2 ? 2 : (h->use_fused ? 32 : h->cell_tile)));
  *face_tile = h->use_fused ? 0 : h->face_tile;
  return DG_OK;
}

int dg_rhs(dg_handle* h, const void* W_dev, void* dWdt_dev, void* stream) {
  if (!check_handle(h) || !W_dev || !dWdt_dev) return DG_ERR_ARG;
  if (W_dev == dWdt_dev) return fail(h, DG_ERR_ARG, "dg_rhs: W and dWdt alias");
  if (check_gravity(h, "dg_rhs") != DG_OK) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return h->prec == DG_FP64 ? rhs_into<double>(h, W_dev, dWdt_dev, s)
                            : rhs_into<float>(h, W_dev, dWdt_dev, s);
}

int dg_compute_dt(dg_handle* h, const void* W_dev, double* dt_dev, void* stream) {
  if (!check_handle(h) || !W_dev || !dt_dev) return DG_ERR_ARG;
  if (check_gravity(h, "dg_compute_dt") != DG_OK) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return h->prec == DG_FP64 ? compute_dt_impl<double>(h, W_dev, dt_dev, s)
                            : compute_dt_impl<float>(h, W_dev, dt_dev, s);
}

int dg_rk_step(dg_handle* h, void* W_dev, double dt, double* dt_used_dev, void* stream) {
  if (!check_handle(h) || !W_dev) return DG_ERR_ARG;
  if (check_gravity(h, "dg_rk_step") != DG_OK) return DG_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return rk_step_dispatch(h, W_dev, dt, dt_used_dev, static_cast<cudaStream_t>(stream));
}

static int advance_graph(dg_handle* h, void* W_dev, int n_steps, double dt, double* dt_hist_dev, cudaStream_t s);
// recorded step graphs kept per handle (dg_advance, dg_advance_dt)
constexpr size_t GRAPH_CACHE_MAX = 64;

int dg_advance(dg_handle* h, void* W_dev, int n_steps, double* dt_hist_dev, void* stream) {
  if (!check_handle(h) || !W_dev || n_steps < 0) return DG_ERR_ARG;
  if (check_gravity(h, "dg_advance") != DG_OK) return DG_ERR_ARG;
  if (n_steps == 0) return DG_OK;
  std::lock_guard<std::mutex> lock(h->mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->advance_mode == DG_ADVANCE_PERSISTENT && persist_supported(h))
    return h->prec == DG_FP64 ? advance_persistent<double>(h, W_dev, n_steps, dt_hist_dev, s)
                              : advance_persistent<float>(h, W_dev, n_steps, dt_hist_dev, s);
  return advance_graph(h, W_dev, n_steps, 0.0, dt_hist_dev, s);
}

int dg_advance_dt(dg_handle* h, void* W_dev, int n_steps, double dt, void* stream) {
  if (!check_handle(h) || !W_dev || n_steps < 0) return DG_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, DG_ERR_ARG, "dg_advance_dt: dt must be positive");
  if (check_gravity(h, "dg_advance_dt") != DG_OK) return DG_ERR_ARG;
  if (n_steps == 0) return DG_OK;
  std::lock_guard<std::mutex> lock(h->mu);
  return advance_graph(h, W_dev, n_steps, dt, nullptr, static_cast<cudaStream_t>(stream));
}

// records n_steps steps into a graph (on the handle's capture stream)
static int capture_steps(dg_handle* h, void* W_dev, int n_steps, double dt, double* dt_hist_dev,
                         cudaGraphExec_t* out) {
  cudaError_t eb = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (eb != cudaSuccess) return cuda_fail(h, eb, "cudaStreamBeginCapture");
  int r = DG_OK;
  for (int i = 0; i < n_steps && r == DG_OK; ++i)
    r = rk_step_dispatch(h, W_dev, dt, dt_hist_dev ? dt_hist_dev + (size_t)i * h->nprob : nullptr, h->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (r != DG_OK) { if (g) cudaGraphDestroy(g); return r; }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaGraphInstantiate"); }
  h->graph_defs.push_back(g);
  return DG_OK;
}

// With profiling on: the steps' graph with an event pair around every kernel
// (event-record nodes), replayed, waited for, and its kernels' device times
// added to the handle's sums.
static int advance_graph_profiled(dg_handle* h, void* W_dev, int n_steps, double dt, double* dt_hist_dev,
                                  cudaStream_t s) {
  auto key = std::make_tuple(W_dev, n_steps, (void*)dt_hist_dev, dt);
  auto it = h->pgraphs.find(key);
  if (it == h->pgraphs.end()) {
    if (h->pgraphs.size() >= GRAPH_CACHE_MAX) drop_graphs(h);
    dg_handle::ProfGraph pg;
    // the capture brackets launches with events of its own pool and marks
    std::swap(h->ev_pool, pg.ev);
    std::swap(h->ev_marks, pg.marks);
    const size_t used = h->ev_used;
    h->ev_used = 0;
    const int r = capture_steps(h, W_dev, n_steps, dt, dt_hist_dev, &pg.exec);
    std::swap(h->ev_pool, pg.ev);
    std::swap(h->ev_marks, pg.marks);
    h->ev_used = used;
    if (r != DG_OK) {
      for (cudaEvent_t e : pg.ev) cudaEventDestroy(e);
      return r;
    }
    it = h->pgraphs.emplace(key, std::move(pg)).first;
  }
  DG_CUDA(h, cudaGraphLaunch(it->second.exec, s));
  DG_CUDA(h, cudaStreamSynchronize(s));
  for (const auto& mk : it->second.marks) {
    float ms = 0.0f;
    DG_CUDA(h, cudaEventElapsedTime(&ms, it->second.ev[mk.second], it->second.ev[mk.second + 1]));
    h->prof_ms[mk.first] += ms;
    h->prof_n[mk.first] += 1;
  }
  return DG_OK;
}

// n_steps steps (dt > 0 fixed, else CFL) as one graph launch, recorded on first use
static int advance_graph(dg_handle* h, void* W_dev, int n_steps, double dt, double* dt_hist_dev, cudaStream_t s) {
  if (h->profiling) return advance_graph_profiled(h, W_dev, n_steps, dt, dt_hist_dev, s);
  auto key = std::make_tuple(W_dev, n_steps, (void*)dt_hist_dev, dt);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    // a bounded cache: callers that vary dt or the buffer every call would
    // otherwise accumulate graphs (an executable graph still in flight is
    // freed when it completes)
    if (h->graphs.size() >= GRAPH_CACHE_MAX) drop_graphs(h);
    cudaGraphExec_t ge = nullptr;
    const int r = capture_steps(h, W_dev, n_steps, dt, dt_hist_dev, &ge);
    if (r != DG_OK) return r;
    it = h->graphs.emplace(key, ge).first;
  }
  DG_CUDA(h, cudaGraphLaunch(it->second, s));
  return DG_OK;
}

int dg_batch_advance(dg_handle* h, void* W_dev, int n_steps, double* dt_hist_dev, void* stream) {
  return dg_advance(h, W_dev, n_steps, dt_hist_dev, stream);
}

int dg_n_problems(const dg_handle* h, int* n_problems, int64_t* cell_offsets_host) {
  if (!check_handle(h) || !n_problems) return DG_ERR_ARG;
  *n_problems = h->nprob;
  if (cell_offsets_host) {
    int64_t off = 0;
    int p = 0;
    cell_offsets_host[0] = 0;
    for (int c = 0; c < h->ncells; ++c) {
      const int pc = h->nprob > 1 ? h->prob[c] : 0;
      while (p < pc) cell_offsets_host[++p] = c;
      off = c + 1;
    }
    while (p < h->nprob) cell_offsets_host[++p] = off;
  }
  return DG_OK;
}

int dg_rk_step_adjoint(dg_handle* h, const void* W_n_dev, double dt, const void* lam_np1_dev,
                       void* lam_n_dev, void* stream) {
  if (!check_handle(h) || !W_n_dev || !lam_np1_dev || !lam_n_dev) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_rk_step_adjoint")) return r;
  if (!(dt > 0.0)) return fail(h, DG_ERR_ARG, "dg_rk_step_adjoint: dt must be positive (frozen)");
  if (h->opt.slope_limiter != DG_LIMITER_NONE || h->opt.positivity)
    return fail(h, DG_ERR_ARG, "dg_rk_step_adjoint: needs an unlimited handle");
  if (h->accel || h->accel_stale)
    return fail(h, DG_ERR_UNSUPPORTED, "dg_rk_step_adjoint: not with a gravity source");
  std::lock_guard<std::mutex> lock(h->mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return h->prec == DG_FP64 ? adjoint_step_impl<double>(h, W_n_dev, dt, lam_np1_dev, lam_n_dev, s)
                            : adjoint_step_impl<float>(h, W_n_dev, dt, lam_np1_dev, lam_n_dev, s);
}

int dg_limit(dg_handle* h, void* W_dev, void* stream) {
  if (!check_handle(h) || !W_dev) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_limit")) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)h->nv * h->N * h->ncells * h->esize;
  void* tmp = h->regs.back();
  DG_CUDA(h, cudaMemcpyAsync(tmp, W_dev, bytes, cudaMemcpyDeviceToDevice, s));
  return h->prec == DG_FP64 ? run_limit<double>(h, tmp, W_dev, s) : run_limit<float>(h, tmp, W_dev, s);
}

int dg_totals(dg_handle* h, const void* W_dev, double* totals_dev, void* stream) {
  if (!check_handle(h) || !W_dev || !totals_dev) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->prec == DG_FP64) {
    AuxArgs<double> a = aux_args<double>(h);
    a.W = static_cast<const double*>(W_dev);
    a.out = totals_dev;
    DG_CUDA(h, h->ks->totals(&a, s));
  } else {
    AuxArgs<float> a = aux_args<float>(h);
    a.W = static_cast<const float*>(W_dev);
    a.out = totals_dev;
    DG_CUDA(h, h->ks->totals(&a, s));
  }
  return DG_OK;
}

int dg_l1_density(dg_handle* h, const void* W_dev, const double* rho_ref_dev, double* out_dev,
                  void* stream) {
  if (!check_handle(h) || !W_dev || !rho_ref_dev || !out_dev) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->prec == DG_FP64) {
    AuxArgs<double> a = aux_args<double>(h);
    a.W = static_cast<const double*>(W_dev);
    a.u = rho_ref_dev;
    a.out = out_dev;
    DG_CUDA(h, h->ks->l1(&a, s));
  } else {
    AuxArgs<float> a = aux_args<float>(h);
    a.W = static_cast<const float*>(W_dev);
    a.u = rho_ref_dev;
    a.out = out_dev;
    DG_CUDA(h, h->ks->l1(&a, s));
  }
  return DG_OK;
}

int dg_node_weights(dg_handle* h, const void* W_dev, void* Wnode_dev, void* stream) {
  if (!check_handle(h) || !W_dev || !Wnode_dev) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_node_weights")) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->prec == DG_FP64) {
    AuxArgs<double> a = aux_args<double>(h);
    a.W = static_cast<const double*>(W_dev);
    a.Wout = static_cast<double*>(Wnode_dev);
    DG_CUDA(h, h->ks->node_weights(&a, s));
  } else {
    AuxArgs<float> a = aux_args<float>(h);
    a.W = static_cast<const float*>(W_dev);
    a.Wout = static_cast<float*>(Wnode_dev);
    DG_CUDA(h, h->ks->node_weights(&a, s));
  }
  return DG_OK;
}

int dg_neighbor_table(const dg_handle* h, int32_t* host_out) {
  if (!check_handle(h) || !host_out) return DG_ERR_ARG;
  if (h->tables_on_device) {
    const size_t n = (size_t)2 * h->dim * h->ncells;
    return cudaMemcpy(host_out, h->md.nbr, n * sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess
               ? DG_OK : DG_ERR_CUDA;
  }
  std::memcpy(host_out, h->nbr.data(), h->nbr.size() * sizeof(int32_t));
  return DG_OK;
}

int dg_cell_levels(const dg_handle* h, int32_t* host_out) {
  if (!check_handle(h) || !host_out) return DG_ERR_ARG;
  if (h->tables_on_device) {
    std::vector<int8_t> lv((size_t)h->ncells);
    if (cudaMemcpy(lv.data(), h->md.level, lv.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_ERR_CUDA;
    for (int c = 0; c < h->ncells; ++c) host_out[c] = lv[c];
    return DG_OK;
  }
  for (int c = 0; c < h->ncells; ++c) host_out[c] = h->level[c];
  return DG_OK;
}

int dg_set_gravity(dg_handle* h, const double* accel_dev, void* stream) {
  if (!check_handle(h)) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_set_gravity")) return r;
  std::lock_guard<std::mutex> lock(h->mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  drop_graphs(h);  // recorded launches carry the old field pointer
  if (!accel_dev) {
    dfree(h, h->accel);
    h->accel = nullptr;
    h->accel_stale = false;
    return DG_OK;
  }
  if (h->nprob != 1 || h->ms || h->use_tc)
    return fail(h, DG_ERR_UNSUPPORTED, "dg_set_gravity: single problems with DG_FP64 or DG_FP32 only");
  const size_t n = (size_t)h->dim * h->ks->Q * h->ncells;
  if (!h->accel) {
    int r = dalloc(h, std::max<size_t>(n, 1) * h->esize, &h->accel);
    if (r != DG_OK) return r;
  }
  DG_CUDA(h, launch_convert(accel_dev, h->accel, n, (int)h->esize, s));
  h->accel_stale = false;
  return DG_OK;
}

int dg_adapt_mark(dg_handle* h, const void* W_dev, double w_t, double alpha, int32_t* flags_host,
                  int64_t* n_cells_new, int64_t* n_changed, void* stream) {
  if (!check_handle(h) || !W_dev) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_adapt_mark")) return r;
  if (!(w_t > 0.0) || !(alpha >= 1.0)) return fail(h, DG_ERR_ARG, "dg_adapt_mark: need w_t > 0 and alpha >= 1");
  std::lock_guard<std::mutex> lock(h->mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int r = ensure_adapt(h);
  if (r != DG_OK) return r;
  const int cur = h->cur;
  DG_CUDA(h, cudaMemsetAsync(h->adapt_info, 0, sizeof(int32_t), s));
  DG_CUDA(h, launch_adapt_criterion(h->bg, W_dev, (int)h->esize, h->N, h->ncells, h->base_first[cur],
                                    h->base_node[cur], h->tab64 + h->ks->off_pref, alpha * w_t, w_t / alpha,
                                    h->adapt_crit, s));
  DG_CUDA(h, launch_adapt_buffer(h->bg, h->adapt_crit, h->base_node[cur], h->adapt_ref, h->adapt_cnt,
                                 h->adapt_info, s));
  return finish_mark(h, flags_host, n_cells_new, n_changed, s);
}

int dg_adapt_set(dg_handle* h, const int32_t* flags_host, int64_t* n_cells_new, int64_t* n_changed,
                 void* stream) {
  if (!check_handle(h) || !flags_host) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_adapt_set")) return r;
  std::lock_guard<std::mutex> lock(h->mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int r = ensure_adapt(h);
  if (r != DG_OK) return r;
  std::vector<uint8_t> fl((size_t)h->bg.nbase);
  for (size_t b = 0; b < fl.size(); ++b) fl[b] = flags_host[b] != 0;
  DG_CUDA(h, cudaMemcpyAsync(h->adapt_ref, fl.data(), fl.size(), cudaMemcpyHostToDevice, s));
  DG_CUDA(h, cudaMemsetAsync(h->adapt_info, 0, sizeof(int32_t), s));
  DG_CUDA(h, launch_adapt_counts(h->bg, h->adapt_ref, h->base_node[h->cur], h->adapt_cnt, h->adapt_info, s));
  return finish_mark(h, nullptr, n_cells_new, n_changed, s);
}

int dg_regrid(dg_handle* h, const void* W_old_dev, void* W_new_dev, void* stream) {
  if (!check_handle(h) || !W_old_dev || !W_new_dev) return DG_ERR_ARG;
  if (int r = tensor_unsupported(h, "dg_regrid")) return r;
  if (W_old_dev == W_new_dev) return fail(h, DG_ERR_ARG, "dg_regrid: W_new must not alias W_old");
  std::lock_guard<std::mutex> lock(h->mu);
  if (!h->mark_pending) return fail(h, DG_ERR_ARG, "dg_regrid: no refinement marked");
  if (h->use_tc && h->next_nodes > 0)
    return fail(h, DG_ERR_UNSUPPORTED, "dg_regrid: tensor-core precisions need a uniform mesh");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = h->dim, cur = h->cur, nxt = 1 - cur;
  const int nc0 = h->ncells;
  const int nc1 = (int)h->next_cells, nn1 = (int)h->next_nodes;
  int r;
  if ((r = ensure_capacity(h, nc1, -1, nn1)) != DG_OK) return r;
  const int64_t L = (int64_t)3 * d * nc1;
  if ((size_t)L + 1 > h->face_cnt_cap) {
    const size_t cap = (size_t)L + L / 4 + 64;
    if ((r = realloc_buf(h, h->face_cnt, cap * sizeof(int32_t))) != DG_OK) return r;
    if ((r = realloc_buf(h, h->face_off, cap * sizeof(int32_t))) != DG_OK) return r;
    h->face_cnt_cap = cap;
  }
  if ((r = ensure_scan_work(h, L)) != DG_OK) return r;
  MeshDev& m = h->md;
  auto level = const_cast<int8_t*>(m.level);
  auto coord = const_cast<int32_t*>(m.coord);
  auto nbr = const_cast<int32_t*>(m.nbr);
  auto sface = const_cast<int32_t*>(m.sface);
  auto scoarse = const_cast<uint8_t*>(m.scoarse);
  auto children = const_cast<int32_t*>(m.node_children);
  DG_CUDA(h, launch_regrid_cells(h->bg, h->base_first[nxt], h->base_node[nxt], nc1, level, coord, children, s));
  DG_CUDA(h, launch_regrid_nbr(h->bg, h->base_first[nxt], h->base_node[nxt], nc1, level, coord, nbr, scoarse,
                               h->face_cnt, s));
  DG_CUDA(h, launch_scan(h->face_cnt, L, h->face_off, h->scan_work, s));
  DG_CUDA(h, launch_adapt_project(h->bg, (int)h->esize, h->nv, h->N, h->tab64 + h->ks->off_pref,
                                  h->base_first[cur], h->base_node[cur], W_old_dev, nc0, level, coord, nc1,
                                  W_new_dev, s));
  int32_t nf1 = 0;
  DG_CUDA(h, cudaMemcpyAsync(&nf1, h->face_off + L, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DG_CUDA(h, cudaStreamSynchronize(s));
  if ((r = ensure_capacity(h, -1, nf1, -1)) != DG_OK) return r;
  DG_CUDA(h, launch_regrid_faces(h->bg, nc1, level, nbr, children, h->face_off, const_cast<int32_t*>(m.fm),
                                 const_cast<int32_t*>(m.fp), const_cast<uint8_t*>(m.finfo), sface, s));
  // the handle now describes the new mesh
  h->ncells = m.ncells = nc1;
  h->nfaces = m.nfaces = nf1;
  h->nnodes = m.nnodes = nn1;
  h->cur = nxt;
  h->mark_pending = false;
  h->tables_on_device = true;
  drop_graphs(h);
  if (h->accel) {  // sampled on the old mesh
    dfree(h, h->accel);
    h->accel = nullptr;
    h->accel_stale = true;
  }
  // adjoint work arrays are sized for the old mesh: allocated again on use
  for (void* p : h->adj) dfree(h, p);
  h->adj.clear();
  dfree(h, h->FG);
  h->FG = nullptr;
  return DG_OK;
}

int dg_profile_begin(dg_handle* h) {
  if (!check_handle(h)) return DG_ERR_ARG;
  h->profiling = true;
  h->ev_used = 0;
  h->ev_marks.clear();
  for (int i = 0; i < DG_KERNEL_KINDS; ++i) { h->prof_ms[i] = 0.0; h->prof_n[i] = 0; }
  return DG_OK;
}

int dg_profile_end(dg_handle* h, int* launches, double* total_ms, int n_kinds) {
  if (!check_handle(h) || n_kinds < 0 || (n_kinds > 0 && (!launches || !total_ms))) return DG_ERR_ARG;
  h->profiling = false;
  for (int i = 0; i < n_kinds; ++i) { launches[i] = 0; total_ms[i] = 0.0; }
  for (const auto& mk : h->ev_marks) {
    DG_CUDA(h, cudaEventSynchronize(h->ev_pool[mk.second + 1]));
    float ms = 0.0f;
    DG_CUDA(h, cudaEventElapsedTime(&ms, h->ev_pool[mk.second], h->ev_pool[mk.second + 1]));
    if (mk.first < n_kinds) {
      launches[mk.first] += 1;
      total_ms[mk.first] += ms;
    }
  }
  h->ev_marks.clear();
  h->ev_used = 0;
  for (int i = 0; i < DG_KERNEL_KINDS; ++i) {  // replays of profiled graphs
    if (i < n_kinds) {
      launches[i] += h->prof_n[i];
      total_ms[i] += h->prof_ms[i];
    }
    h->prof_ms[i] = 0.0;
    h->prof_n[i] = 0;
  }
  return DG_OK;
}

int dg_set_advance_mode(dg_handle* h, int mode) {
  if (!check_handle(h)) return DG_ERR_ARG;
  if (mode != DG_ADVANCE_GRAPH && mode != DG_ADVANCE_PERSISTENT) return fail(h, DG_ERR_ARG, "dg_set_advance_mode: mode");
  if (mode == DG_ADVANCE_PERSISTENT && !persist_supported(h))
    return fail(h, DG_ERR_UNSUPPORTED,
                "dg_set_advance_mode: the persistent step kernel needs a 2D FP64 or FP32 handle with the "
                "CUDA-core stage kernels, no gravity source and at most 5 stages");
  std::lock_guard<std::mutex> lock(h->mu);
  h->advance_mode = mode;
  return DG_OK;
}

int dg_advance_mode(const dg_handle* h, int* mode) {
  if (!check_handle(h) || !mode) return DG_ERR_ARG;
  *mode = h->advance_mode == DG_ADVANCE_PERSISTENT && persist_supported(h) ? DG_ADVANCE_PERSISTENT
                                                                           : DG_ADVANCE_GRAPH;
  return DG_OK;
}

int dg_set_overlap(dg_handle* h, int on) {
  if (!check_handle(h)) return DG_ERR_ARG;
  if (on != 0 && on != 1) return fail(h, DG_ERR_ARG, "dg_set_overlap: on must be 0 or 1");
  std::lock_guard<std::mutex> lock(h->mu);
  h->pdl = on;
  drop_graphs(h);  // recorded launches carry the old launch attributes
  return DG_OK;
}

int dg_overlap(const dg_handle* h, int* on) {
  if (!check_handle(h) || !on) return DG_ERR_ARG;
  *on = h->pdl;
  return DG_OK;
}

int dg_test_flux_math(int op, const double* x_dev, double* out_dev, int64_t n, void* stream) {
  if (op < 0 || op > 3 || !x_dev || !out_dev || n < 0) return DG_ERR_ARG;
  return launch_flux_math(op, x_dev, out_dev, n, static_cast<cudaStream_t>(stream)) == cudaSuccess ? DG_OK
                                                                                                : DG_ERR_CUDA;
}

int dg_test_mesh_tables(const dg_mesh_desc* meshes, int n_problems, int64_t* counts, int32_t* nbr,
                        int32_t* levels, int32_t* faces, int32_t* sface, int32_t* prob) {
  if (!meshes || !counts || n_problems < 1) return DG_ERR_ARG;
  if (meshes[0].dim != 2 && meshes[0].dim != 3) return DG_ERR_ARG;
  // a handle without device state: the builders are host work only
  dg_handle h;
  h.dim = meshes[0].dim;
  const int r = n_problems == 1 ? build_mesh(&h, meshes) : build_batch(&h, meshes, n_problems);
  if (r != DG_OK) return r;
  const size_t nc = (size_t)h.ncells, nf = (size_t)h.nfaces, sides = (size_t)2 * h.dim;
  counts[0] = (int64_t)nc;
  counts[1] = (int64_t)nf;
  counts[2] = (int64_t)h.nnodes;
  if (nbr) std::copy(h.nbr.begin(), h.nbr.end(), nbr);
  if (levels)
    for (size_t c = 0; c < nc; ++c) levels[c] = h.level[c];
  if (faces)
    for (size_t f = 0; f < nf; ++f) {
      faces[f] = h.fm[f];
      faces[nf + f] = h.fp[f];
      faces[2 * nf + f] = h.finfo[f];
    }
  if (sface) std::copy(h.sface.begin(), h.sface.begin() + sides * nc, sface);
  if (prob)
    for (size_t c = 0; c < nc; ++c) prob[c] = n_problems == 1 ? 0 : h.prob[c];
  return DG_OK;
}

static_assert(MAX_IN == 4 && MAX_OUT == 3 && DG_TEST_OP_DOUBLES == 5 + MAX_IN + MAX_OUT + MAX_OUT * MAX_IN + MAX_OUT,
              "dg_test_stage_program record layout");

int dg_test_stage_program(int rk_order, int limited, double* ops_out, int max_ops, int* n_ops, int* n_regs) {
  if (rk_order < 1 || rk_order > 4 || (limited != 0 && limited != 1) || !n_ops || !n_regs || max_ops < 0)
    return DG_ERR_ARG;
  Program P;
  std::string err;
  if (!build_program(rk_order, limited == 1, P, err)) return DG_ERR_ARG;
  *n_ops = (int)P.ops.size();
  *n_regs = P.n_phys;
  if (!ops_out) return DG_OK;
  if (max_ops < (int)P.ops.size()) return DG_ERR_ARG;
  for (size_t i = 0; i < P.ops.size(); ++i) {
    const Op& op = P.ops[i];
    double* r = ops_out + i * DG_TEST_OP_DOUBLES;
    r[0] = op.in_reg;
    r[1] = op.n_in;
    r[2] = op.n_out;
    r[3] = op.lim_src;
    r[4] = op.lim_dst;
    for (int j = 0; j < MAX_IN; ++j) r[5 + j] = j < op.n_in ? op.in[j] : -1;
    for (int o = 0; o < MAX_OUT; ++o) r[9 + o] = o < op.n_out ? op.out[o] : -1;
    for (int o = 0; o < MAX_OUT; ++o)
      for (int j = 0; j < MAX_IN; ++j) r[12 + 4 * o + j] = op.C[o][j];
    for (int o = 0; o < MAX_OUT; ++o) r[24 + o] = op.ck[o];
  }
  return DG_OK;
}

int dg_test_force_timeout(dg_handle* h) {
  if (!check_handle(h)) return DG_ERR_ARG;
  if (!h->use_tc) return fail(h, DG_ERR_UNSUPPORTED, "dg_test_force_timeout: no tensor-core cell kernel");
  h->tc_hook = 1;
  return DG_OK;
}

int dg_status(dg_handle* h, int* device_status_host) {
  if (!check_handle(h) || !device_status_host) return DG_ERR_ARG;
  int bits = 0;
  DG_CUDA(h, cudaMemcpy(&bits, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  DG_CUDA(h, cudaMemset(h->status, 0, sizeof(int)));
  int code = DG_OK;
  if (bits & (1 << DG_ERR_NONPHYSICAL_BIT)) code = DG_ERR_NONPHYSICAL;
  else if (bits & (1 << DG_ERR_TIMEOUT_BIT)) code = DG_ERR_TIMEOUT;
  *device_status_host = code;
  return DG_OK;
}

}  // extern "C"
