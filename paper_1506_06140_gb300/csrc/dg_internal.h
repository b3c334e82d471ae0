// Internal interfaces of libdg: device-side table layouts, kernel argument
// blocks and the per-(precision, dim, k) kernel set.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace dgi {

// ---------------------------------------------------------------------------
// Compile-time sizes of a (dim, k) scheme.  B = 0: the paper's basis of
// total degree <= k; B = 1: the tensor-product basis Q_k (every exponent
// <= k, (k+1)^dim functions; 2D kernels only).
template <int DIM, int K, int B = 0>
struct Shape {
  static constexpr int N = B ? (DIM == 2 ? (K + 1) * (K + 1) : (K + 1) * (K + 1) * (K + 1))
                             : (DIM == 2 ? (K + 1) * (K + 2) / 2 : (K + 1) * (K + 2) * (K + 3) / 6);
  static constexpr int NV = DIM + 2;
  static constexpr int K1 = K + 1;
  static constexpr int Q = DIM == 2 ? K1 * K1 : K1 * K1 * K1;          // volume points
  static constexpr int QF = DIM == 2 ? K1 : K1 * K1;                   // face points
  static constexpr int K3 = K + 3;
  static constexpr int Q1 = DIM == 2 ? K3 * K3 : K3 * K3 * K3;         // L1-error points
  static constexpr int NSIDE = 2 * DIM;
  static constexpr int NSUB = 1 << (DIM - 1);                          // sub-faces of a face
  static constexpr int NVAR = 1 + NSUB;                                // face point variants
  static constexpr int NCH = 1 << DIM;                                 // children of a node
  static constexpr int M = (K + 4) / 2 < 2 ? 2 : (K + 4) / 2;          // Lobatto points, m >= (k+3)/2
  static constexpr int MF = DIM == 2 ? M : M * K1;                     // points of one S_a per ... (unused)
  static constexpr int NSP = DIM * M * QF;                             // |S| (eq. union_quad_points)
  // offsets into the per-handle table (elements)
  static constexpr int OFF_PHI = 0;                                    // [Q][N]     phi_l(xi_q)
  static constexpr int OFF_DPHIW = OFF_PHI + Q * N;                    // [DIM][Q][N] dphi_l/dxi_a * w_q
  static constexpr int OFF_PHIF = OFF_DPHIW + DIM * Q * N;             // [NSIDE][NVAR][QF][N] phi at face points
  static constexpr int OFF_PHIFW = OFF_PHIF + NSIDE * NVAR * QF * N;   // same, * w_q (* 2^-(d-1) for sub-faces)
  static constexpr int OFF_PREF = OFF_PHIFW + NSIDE * NVAR * QF * N;   // [NCH][N][N] refinement matrices (j,l)
  static constexpr int OFF_PROJ = OFF_PREF + NCH * N * N;              // [Q][N] phi * w_q * 2^-d
  static constexpr int OFF_SPHI = OFF_PROJ + Q * N;                    // [NSP][N] phi at the set S
  static constexpr int OFF_L1PHI = OFF_SPHI + NSP * N;                 // [Q1][N]  phi at L1 points
  static constexpr int OFF_L1W = OFF_L1PHI + Q1 * N;                   // [Q1]     L1 weights
  static constexpr int OFF_XI = OFF_L1W + Q1;                          // [Q][3]   volume points
  static constexpr int OFF_XI1 = OFF_XI + Q * 3;                       // [Q1][3]  L1 points
  static constexpr int OFF_DEG = OFF_XI1 + Q1 * 3;                     // [N]      degree of phi_l
  static constexpr int OFF_PMAX = OFF_DEG + N;                         // [N] max |phi_l| on [-1,1]^d
  static constexpr int OFF_1D = OFF_PMAX + N;                          // Tab1D (sizes of Tab1D<double>)
  static constexpr int TAB_SIZE = OFF_1D + 156;
  // values per variable and face in the face-flux array: the flux at the
  // face's Gauss points (2D), or its moments against the face's Legendre
  // products of total degree <= k (3D, eq. dg_term3 restricted to a face)
  static constexpr int NM = K1 * (K1 + 1) / 2;
  static constexpr int FV = DIM == 3 ? NM : QF;
};

// One-dimensional tables of the tensor-product Gauss rule (k+1 <= 4 nodes),
// passed by value inside the kernel arguments so that, with all loops
// unrolled, every table entry is an immediate constant-bank operand.
template <typename real>
struct Tab1D {
  real P[4][4];      // P[a][i]  = sqrt(2a+1) P_a(x_i)
  real PW[4][4];     // PW[a][i] = P[a][i] w_i
  real DW[4][4];     // DW[a][i] = sqrt(2a+1) P_a'(x_i) w_i
  real PH[2][4][4];  // PH[h][a][i] = sqrt(2a+1) P_a((x_i + 2h - 1) / 2): node i of half h
  real PWH[2][4][4]; // PWH[h][a][i] = PH[h][a][i] w_i
  real PE[2][4];     // PE[s][a] = sqrt(2a+1) P_a(2s - 1): values at -1 (s=0) and +1 (s=1)
  real W[4];         // Gauss weights w_i
  real TH[2][4][4];  // TH[h][a][b]: P~_a((x + 2h - 1) / 2) = sum_{b <= a} TH[h][a][b] P~_b(x)
};

// ---------------------------------------------------------------------------
// Device mesh tables (all arrays owned by the handle).
struct MeshDev {
  int ncells = 0, nfaces = 0, nnodes = 0;
  double dx0 = 1.0;            // base edge length
  double lo[3] = {0, 0, 0};
  int n[3] = {1, 1, 1};
  const int8_t* level = nullptr;         // [ncells]
  const int32_t* coord = nullptr;        // [3][ncells] integer position at the cell's level
  const int32_t* nbr = nullptr;          // [2*dim][ncells]
  const int32_t* fm = nullptr;           // [nfaces] minus-side cell, -1 = mirror of the plus side
  const int32_t* fp = nullptr;           // [nfaces] plus-side cell, -1 = mirror of the minus side
  const uint8_t* finfo = nullptr;        // [nfaces] dir | vm << 2 | vp << 5
  const int32_t* sface = nullptr;        // [2*dim][ncells] first face entry of each side
  const uint8_t* scoarse = nullptr;      // [ncells] bit s: side s holds NSUB sub-face entries
  const int32_t* node_children = nullptr;// [nnodes][2^dim]
  // ensembles of independent problems (all nullptr for a single problem)
  int nprob = 1;
  const int32_t* prob = nullptr;         // [ncells] problem of the cell
  const double* dx_prob = nullptr;       // [nprob] base edge length
  const double* lo_prob = nullptr;       // [nprob][3] domain origin
};

__host__ __device__ __forceinline__ int cell_problem(const MeshDev& m, int c) {
  return m.prob ? m.prob[c] : 0;
}

// bits of the device status word
constexpr int DG_ERR_NONPHYSICAL_BIT = 4;
constexpr int DG_ERR_TIMEOUT_BIT = 5;

constexpr int MAX_IN = 4;
constexpr int MAX_OUT = 3;

// One stage: face fluxes of U, then per cell
//   out_o = sum_r C[o][r] in_r + ck[o] * dt * dWdt(U)
template <typename real>
struct StageArgs {
  MeshDev m;
  Tab1D<real> t1;
  real pre[2] = {0, 0};         // 2^(1-d) / dx per refinement level
  const real* pre_prob = nullptr;  // [nprob] 2^(1-d) / dx per problem (ensembles)
  const real* tab = nullptr;
  const real* U = nullptr;
  real* F = nullptr;            // face fluxes [NV][FV][nfaces]: point values (2D), moments (3D)
  double gamma = 1.4;
  real gam = real(1.4), gm1 = real(0.4);  // gamma and gamma - 1 in the state precision (set on the host)
  int n_in = 0, n_out = 0;
  const real* in[MAX_IN] = {nullptr, nullptr, nullptr, nullptr};
  real* out[MAX_OUT] = {nullptr, nullptr, nullptr};
  real C[MAX_OUT][MAX_IN] = {};
  real ck[MAX_OUT] = {};
  const double* dt = nullptr;   // device timestep per problem; nullptr means dt = 1
  int cell_tile = 0;            // cells per block of the cell kernel (0: its default)
  const void* dtab = nullptr;   // host copy of the one-thread-per-cell kernel's tables
  int face_tile = 0;            // faces per block of the face kernel (0: its default)
  const real* tcB = nullptr;    // tensor-core B operands (tensor-core cell kernel)
  int* status = nullptr;        // device status word
  int tc_hook = 0;              // test hook of the tensor-core cell kernel: 1 = its first CTA skips
                                // its first MMA and commit and waits with a short limit
  const real* accel = nullptr;  // [DIM][Q][ncells] external acceleration at the volume points
                                // (gravity source, eq. gravity_term); nullptr: none
  int pdl = 0;                  // 1: launched as a programmatic dependent of the previous kernel
};

// Stage arguments of the mixed-precision kernels (FP64 state, FP32
// right-hand side in perturbation form).
struct MixedArgs {
  StageArgs<double> a;  // mesh, FP64 state, stage program, timesteps
  Tab1D<float> t;       // the 1D tables in FP32
  float* G = nullptr;   // [NV][QF][nfaces] F* - f(ubar_m), m the face's minus cell
  float* D = nullptr;   // [NV][nfaces]     f(ubar_m) - f(ubar_p)
  // Delta registers (unlimited stage programs): every stage state is
  // U = W + R with W = a.U the FP64 state and R an FP32 register.
  const float* R = nullptr;          // delta of the evaluated state (nullptr: U = W)
  int delta = 0;                     // 1: the epilogue combines delta registers
  int n_inR = 0;                     // inputs other than W
  const float* inR[MAX_IN] = {};     // their deltas
  float Cf[MAX_IN] = {};             // their coefficients
  float ckf = 0.0f;                  // coefficient of dt dW/dt
  float gamf = 1.4f, g1f = 0.4f;     // gamma and gamma - 1 in FP32 (set on the host)
  float* outR = nullptr;             // output delta; nullptr: W += increment (a.out[0] = W)
  // FP32 split of W within a step: Wf = W rounded (weight 0 truncated) and
  // Wlo = the rest of weight 0.  wf_mode 1: the cell kernel writes them (first
  // stage); 2: both kernels read them instead of W; 0: unused.
  int wf_mode = 0;
  float* Wf = nullptr;               // [NV][N][ncells]
  float* Wlo = nullptr;              // [NV][ncells]
  const float* tcB = nullptr;        // tensor-core B operands (DG_MIXED_TC)
};

template <typename real>
struct LimitArgs {
  MeshDev m;
  int pdl = 0;  // 1: launched as a programmatic dependent of the previous kernel
  const double* tab64 = nullptr;  // FP64 tables (same layout)
  const real* tabr = nullptr;     // the same tables in the state precision
  const float* tab32 = nullptr;   // the same tables in FP32 (positivity precheck)
  const real* Uin = nullptr;
  real* Uout = nullptr;
  double gamma = 1.4;
  int limiter = 0;
  double beta = 1.0, Mtilde = 0.5;
  int positivity = 0;
  double eps = 1e-10;
  int fp32_slopes = 0;            // FP64 state: run the slope limiter on FP32-rounded values
  unsigned long long* counts = nullptr;  // [3] cells changed by the slope / positivity limiter, FP64-pass cells
  int* queue = nullptr;          // [ncells] cells left to the positivity pass
  int* queue_len = nullptr;      // their number
  int* status = nullptr;
};

template <typename real>
struct AuxArgs {
  MeshDev m;
  int pdl = 0;  // 1: launched as a programmatic dependent of the previous kernel
  const double* tab64 = nullptr;
  const real* W = nullptr;
  real* Wout = nullptr;
  const double* u = nullptr;      // point values (projection) / reference density (L1)
  double* out = nullptr;          // coordinates / reduction results
  double* partial = nullptr;      // reduction partials
  int nblocks = 0;
  double gamma = 1.4;
  double dt_factor = 1.0;         // CFL factor of the timestep formula
  double volume = 1.0;            // domain volume (L1)
  double inv_dx[2] = {1.0, 1.0};  // 1 / edge length per refinement level
  const double* inv_dx_prob = nullptr;  // [nprob] 1 / base edge length (ensembles)
  unsigned long long* dt_bits = nullptr;
  int* status = nullptr;
  const real* accel = nullptr;    // [DIM][Q][ncells] external acceleration (gravity timestep bound)
  double grav_factor = 0.0;       // dt_factor * sqrt(2 gamma (gamma - 1))
  // timestep finished in the dt kernel itself (nullptr: a separate finalize):
  // the last block turns dt_bits into dt_out = dt_factor / speed and resets
  // dt_bits and dt_done for the next launch
  double* dt_out = nullptr;       // [nprob]
  double* dt_copy = nullptr;      // [nprob] optional second copy
  unsigned int* dt_done = nullptr;  // blocks finished
};

// Adjoint of one stage: given the stage state U and a cotangent G on dWdt(U),
// accumulate lam += J(U)^T G into the 'acc' array (same layout as W).
template <typename real>
struct AdjointArgs {
  MeshDev m;
  Tab1D<real> t1;
  real pre[2] = {0, 0};          // 2^(1-d) / dx per refinement level
  const real* pre_prob = nullptr;  // [nprob] per problem (ensembles)
  const real* U = nullptr;       // state at which dW/dt is linearised
  const real* G = nullptr;       // cotangent of dW/dt (layout of W)
  real* FG = nullptr;            // face cotangents of the traces [2 sides][NV][QF][nfaces]
  real* acc = nullptr;           // output: acc = scale * J(U)^T G
  double gamma = 1.4;
  double scale = 1.0;
};

// Plan of the persistent whole-step kernel (dg_persist.cuh): the arguments
// of every phase of one RK step, in device memory.  Records are 16-byte
// aligned (the kernel copies them into shared memory in 16-byte chunks).
constexpr int PERSIST_MAX_OPS = 5;

template <typename real>
struct PersistOp {
  alignas(16) StageArgs<real> st;  // face and cell phases
  alignas(16) LimitArgs<real> la;  // limiter phases (lim != 0)
  int lim = 0;
};

template <typename real>
struct PersistPlan {
  PersistOp<real> op[PERSIST_MAX_OPS];
  alignas(16) AuxArgs<real> dt;    // timestep phase; dt_copy (if set) advances by nprob per step
  int n_ops = 0;
  int face_blocks = 0, cell_blocks = 0, lim_blocks = 0, pos_blocks = 0, dt_blocks = 0;
};

// out = sum_r c[r] x[r] over n elements (x[r] may alias out)
constexpr int MAX_COMBINE = 8;
template <typename real>
struct CombineArgs {
  real* out = nullptr;
  const real* x[MAX_COMBINE] = {};
  real c[MAX_COMBINE] = {};
  int n_terms = 0;
  size_t n = 0;
};

// Kernel set of one (precision, dim, k).
struct KernelSet {
  int dim = 0, k = 0, prec = 0, basis = 0;  // basis: 0 total degree <= k, 1 tensor product Q_k
  int N = 0, NV = 0, Q = 0, QF = 0, Q1 = 0, NSUB = 0, NSP = 0, M = 0, tab_size = 0;
  int off_pref = 0;  // offset of the refinement matrices in the table
  // host: fill the table (double) from 1D Gauss and Lobatto rules
  void (*fill_tables)(std::vector<double>& tab, const std::vector<double>& gx,
                      const std::vector<double>& gw, const std::vector<double>& g3x,
                      const std::vector<double>& g3w, const std::vector<double>& lx) = nullptr;
  cudaError_t (*prepare)() = nullptr;  // one-time kernel attributes (not capturable)
  // tiles of the stage kernels: default and largest cells / faces per block
  int cell_tile = 32, cell_tile_max = 32, face_tile = 32, face_tile_max = 32;
  cudaError_t (*face)(const void* stage_args, cudaStream_t s) = nullptr;
  cudaError_t (*cell)(const void* stage_args, cudaStream_t s) = nullptr;
  cudaError_t (*limit)(const void* limit_args, cudaStream_t s) = nullptr;
  cudaError_t (*project)(const void* aux, cudaStream_t s) = nullptr;
  cudaError_t (*points)(const void* aux, int l1rule, cudaStream_t s) = nullptr;
  cudaError_t (*dt)(const void* aux, cudaStream_t s) = nullptr;
  cudaError_t (*totals)(const void* aux, cudaStream_t s) = nullptr;
  cudaError_t (*l1)(const void* aux, cudaStream_t s) = nullptr;
  cudaError_t (*node_weights)(const void* aux, cudaStream_t s) = nullptr;
  cudaError_t (*adj_face)(const void* adj_args, cudaStream_t s) = nullptr;
  cudaError_t (*adj_cell)(const void* adj_args, cudaStream_t s) = nullptr;
  cudaError_t (*combine)(const void* combine_args, cudaStream_t s) = nullptr;
  // packed-pair FP32 cell kernel (2D: two variables per thread), nullptr where not built
  cudaError_t (*cell_x2)(const void* stage_args, cudaStream_t s) = nullptr;
  // one-thread-per-cell FP32 cell kernel (2D), nullptr where not built
  cudaError_t (*cell_direct)(const void* stage_args, cudaStream_t s) = nullptr;
  void (*fill_direct)(const std::vector<double>& tab, std::vector<unsigned char>& out) = nullptr;
  // tensor-core cell kernel (FP32 state, 2D, k = 1..3), nullptr where not built
  cudaError_t (*cell_tc)(const void* stage_args, cudaStream_t s) = nullptr;
  cudaError_t (*prepare_tc)() = nullptr;
  void (*fill_tc)(const std::vector<double>& tab, std::vector<float>& out) = nullptr;
  // fused face + cell kernel (2D uniform meshes), nullptr where not built
  cudaError_t (*stage_fused)(const void* stage_args, cudaStream_t s) = nullptr;
  cudaError_t (*prepare_fused)() = nullptr;
  // persistent whole-step kernel (2D), nullptr where not built: n_steps steps
  // of the plan (a PersistPlan<real> in device memory) in one cooperative
  // launch of at most max_phase_blocks blocks; bar: 3 zeroed words
  cudaError_t (*persist)(const void* plan_dev, int max_phase_blocks, int n_steps, unsigned* bar, int* status,
                         cudaStream_t s) = nullptr;
  cudaError_t (*prepare_persist)() = nullptr;
};

const KernelSet* kernel_set(int prec, int dim, int k, int basis = 0);

// Stage kernels for an FP64 state with an FP32 right-hand side in
// perturbation form (argument block MixedArgs, dg_mixed.cuh).
struct MixedSet {
  int cell_tile = 32, cell_tile_max = 32, face_tile = 32, face_tile_max = 32;
  cudaError_t (*face)(const void* mixed_args, cudaStream_t s) = nullptr;
  cudaError_t (*cell)(const void* mixed_args, cudaStream_t s) = nullptr;
  cudaError_t (*prepare)() = nullptr;
  // tensor-core cell kernel (2D, k = 1..3), nullptr where not built
  cudaError_t (*cell_tc)(const void* mixed_args, cudaStream_t s) = nullptr;
  cudaError_t (*prepare_tc)() = nullptr;
  void (*fill_tc)(const std::vector<double>& tab, std::vector<float>& out) = nullptr;
};

const MixedSet* mixed_set(int dim, int k);

// ---------------------------------------------------------------------------
// Mesh adaptation on the device (dg_regrid.cu).  Base cells are numbered
// lexicographically; first[b] is the first cell of base cell b (first[nbase]
// = the cell count), node_of[b] its node index or -1 for a leaf.
struct BaseGrid {
  int dim = 2, nbase = 0;
  int n[3] = {1, 1, 1};
  int periodic[3] = {1, 1, 1};
};

// criterion per base cell (eqs. cell_ref, node_ref): crit[b] = 1 when the
// largest density slope weight of the leaf exceeds thr_leaf, or that of the
// node weights of a node exceeds thr_node
cudaError_t launch_adapt_criterion(const BaseGrid& g, const void* W, int esize, int N, int ncells,
                                   const int32_t* first, const int32_t* node_of, const double* P,
                                   double thr_leaf, double thr_node, uint8_t* crit, cudaStream_t s);
// one buffer layer: refined[b] = any crit in the 3^d block around b (periodic
// axes wrap); cnt[b] = cells of base cell b on the new mesh; *changed counts
// the base cells whose refinement differs from node_of's
cudaError_t launch_adapt_buffer(const BaseGrid& g, const uint8_t* crit, const int32_t* node_of,
                                uint8_t* refined, int32_t* cnt, int32_t* changed, cudaStream_t s);
// cnt[b] from given flags (refined[b] != 0), with the same change count
cudaError_t launch_adapt_counts(const BaseGrid& g, const uint8_t* refined, const int32_t* node_of,
                                int32_t* cnt, int32_t* changed, cudaStream_t s);
// out[i] = sum_{j<i} in[j] for i <= n (out[n] = the total); work: scan_work_ints(n) ints
cudaError_t launch_scan(const int32_t* in, int64_t n, int32_t* out, int32_t* work, cudaStream_t s);
size_t scan_work_ints(int64_t n);
// cell tables of the new mesh from first[] (node_of[] is derived and written)
cudaError_t launch_regrid_cells(const BaseGrid& g, const int32_t* first, int32_t* node_of, int ncells,
                                int8_t* level, int32_t* coord, int32_t* node_children, cudaStream_t s);
// neighbour table and coarse-side bits; face counts per (axis, cell) then per
// (axis, cell, side) in the numbering of the host mesh builder
cudaError_t launch_regrid_nbr(const BaseGrid& g, const int32_t* first, const int32_t* node_of, int ncells,
                              const int8_t* level, const int32_t* coord, int32_t* nbr, uint8_t* scoarse,
                              int32_t* face_cnt, cudaStream_t s);
cudaError_t launch_regrid_faces(const BaseGrid& g, int ncells, const int8_t* level, const int32_t* nbr,
                                const int32_t* node_children, const int32_t* face_off, int32_t* fm,
                                int32_t* fp, uint8_t* finfo, int32_t* sface, cudaStream_t s);
// the state on the new mesh (Secs. 4.4, 4.5): copy, P_c w, or 2^-d sum_c P_c^T w^c
cudaError_t launch_adapt_project(const BaseGrid& g, int esize, int nv, int N, const double* P,
                                 const int32_t* first0, const int32_t* node0, const void* Wold, int ncells0,
                                 const int8_t* level1, const int32_t* coord1, int ncells1, void* Wnew,
                                 cudaStream_t s);

// shared helper kernels (dg_common.cu)
cudaError_t launch_set_scalar(double* dst, int n, double value, cudaStream_t s);
// dst[i] = value for i < n, elements of esize bytes (4: float, 8: double)
cudaError_t launch_fill(void* dst, size_t n, double value, int esize, cudaStream_t s);
cudaError_t launch_flux_math(int op, const double* x, double* out, int64_t n, cudaStream_t s);
// dst[i] = src[i] converted to elements of esize bytes (4: float, 8: double)
cudaError_t launch_convert(const double* src, void* dst, size_t n, int esize, cudaStream_t s);
cudaError_t launch_dt_finalize(const unsigned long long* bits, int nprob, double factor, double* dt,
                               double* dt_copy, cudaStream_t s);

}  // namespace dgi
