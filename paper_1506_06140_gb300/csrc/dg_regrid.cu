// Mesh adaptation of the two-level mesh on the device (Secs. 4.1, 4.3-4.5).
//
// After an RK step every base cell is checked: a leaf is refined when its
// largest density slope weight |w_rho,1+a| exceeds alpha w_t (eq. cell_ref),
// a node stays refined while the largest slope of its node weights exceeds
// w_t / alpha (eq. node_ref); one layer of base cells around each flagged
// cell is refined as a buffer (Sec. 4.1).  The new numbering (every base cell
// owns one cell or 2^d consecutive children, in base-cell order) comes from
// prefix sums; the cell, neighbour and face tables are then written in
// parallel in the same order as the host mesh builder, and the state is
// carried over by copying unchanged cells, refining with the matrices P_c
// (eq. ref_weights) and merging with 2^-d sum_c P_c^T w^c (eq. deref_weights).
#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dgi {

namespace {

constexpr int RG_THREADS = 256;

__host__ __device__ inline int grid_for(int64_t n, int threads = RG_THREADS) {
  return (int)((n + threads - 1) / threads);
}

__device__ inline void base_coord(const BaseGrid& g, int b, int p[3]) {
  p[0] = b % g.n[0];
  p[1] = (b / g.n[0]) % g.n[1];
  p[2] = b / (g.n[0] * g.n[1]);
}

template <typename real>
__global__ void adapt_criterion_kernel(const BaseGrid g, const real* __restrict__ W, int N, int nc,
                                 const int32_t* __restrict__ first, const int32_t* __restrict__ node_of,
                                 const double* __restrict__ P, double thr_leaf, double thr_node,
                                 uint8_t* __restrict__ crit) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nbase) return;
  const int c0 = first[b];
  const int d = g.dim, nch = 1 << d;
  double slope = 0.0;
  if (node_of[b] < 0) {
    // density (variable 0) slope weights of the leaf: W[0][1 + a][c0]
    for (int a = 0; a < d; ++a) slope = fmax(slope, fabs((double)W[(size_t)(1 + a) * nc + c0]));
    crit[b] = slope > thr_leaf;
  } else {
    // node weights' slope rows, 2^-d sum_c sum_l P_c[l][1+a] w^c_l, summed in
    // child-major order without contraction
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int ch = 0; ch < nch; ++ch)
        for (int l = 0; l < N; ++l)
          s = __dadd_rn(s, __dmul_rn(P[((size_t)ch * N + l) * N + 1 + a], (double)W[(size_t)l * nc + c0 + ch]));
      slope = fmax(slope, fabs(scalbn(s, -d)));
    }
    crit[b] = slope > thr_node;
  }
}

__global__ void adapt_buffer_kernel(const BaseGrid g, const uint8_t* __restrict__ crit,
                              const int32_t* __restrict__ node_of, uint8_t* __restrict__ refined,
                              int32_t* __restrict__ cnt, int32_t* __restrict__ changed) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nbase) return;
  int p[3];
  base_coord(g, b, p);
  const int dz = g.dim == 3 ? 1 : 0;
  int any = 0;
  for (int z = -dz; z <= dz; ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        const int off[3] = {x, y, z};
        int q[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
          q[a] = p[a] + off[a];
          if (q[a] < 0 || q[a] >= g.n[a]) {
            if (a < g.dim && g.periodic[a]) q[a] = (q[a] + g.n[a]) % g.n[a];
            else inside = false;
          }
        }
        if (inside) any |= crit[q[0] + g.n[0] * (q[1] + g.n[1] * q[2])];
      }
  refined[b] = (uint8_t)any;
  cnt[b] = any ? (1 << g.dim) : 1;
  if (any != (node_of[b] >= 0 ? 1 : 0)) atomicAdd(changed, 1);
}

__global__ void adapt_counts_kernel(const BaseGrid g, const uint8_t* __restrict__ refined,
                              const int32_t* __restrict__ node_of, int32_t* __restrict__ cnt,
                              int32_t* __restrict__ changed) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nbase) return;
  const int r = refined[b] ? 1 : 0;
  cnt[b] = r ? (1 << g.dim) : 1;
  if (r != (node_of[b] >= 0 ? 1 : 0)) atomicAdd(changed, 1);
}

// ---- exclusive prefix sum of int32 (three passes over blocks of 2048) ----
constexpr int SC_T = 256, SC_V = 8, SC_B = SC_T * SC_V;

__device__ inline int block_exclusive(int v, int* total) {
  __shared__ int warp_sum[SC_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < SC_T / 32 ? warp_sum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SC_T / 32) warp_sum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int before = (wid > 0 ? warp_sum[wid - 1] : 0) + x - v;
  *total = warp_sum[SC_T / 32 - 1];
  __syncthreads();  // warp_sum is reused by the next call
  return before;
}

__global__ void regrid_scan_reduce_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * SC_B;
  int s = 0;
  for (int i = threadIdx.x; i < SC_B; i += SC_T)
    if (base + i < n) s += in[base + i];
  int total;
  block_exclusive(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// one block: exclusive scan of the block sums in place; *grand = their total
__global__ void regrid_scan_blocks_kernel(int32_t* __restrict__ bsum, int nb, int32_t* __restrict__ grand) {
  int carry = 0;
  for (int base = 0; base < nb; base += SC_T) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    int total;
    const int before = block_exclusive(v, &total);
    if (i < nb) bsum[i] = carry + before;
    carry += total;
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void regrid_scan_down_kernel(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ bsum,
                                 int32_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * SC_B + (int64_t)threadIdx.x * SC_V;
  int v[SC_V];
  int s = 0;
#pragma unroll
  for (int j = 0; j < SC_V; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    s += v[j];
  }
  int total;
  int run = bsum[blockIdx.x] + block_exclusive(s, &total);
#pragma unroll
  for (int j = 0; j < SC_V; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
}

// ---- tables of the new mesh ----
__global__ void regrid_cells_kernel(const BaseGrid g, const int32_t* __restrict__ first, int32_t* __restrict__ node_of,
                             int nc, int8_t* __restrict__ level, int32_t* __restrict__ coord,
                             int32_t* __restrict__ node_children) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nbase) return;
  const int d = g.dim, nch = 1 << d;
  const int f = first[b];
  const bool refined = first[b + 1] - f > 1;
  // every refined base cell before b added nch - 1 cells
  const int node = refined ? (f - b) / (nch - 1) : -1;
  node_of[b] = node;
  int p[3];
  base_coord(g, b, p);
  if (!refined) {
    level[f] = 0;
    coord[f] = p[0];
    coord[(size_t)nc + f] = p[1];
    coord[(size_t)2 * nc + f] = p[2];
    return;
  }
  for (int ch = 0; ch < nch; ++ch) {
    const int c = f + ch;
    level[c] = 1;
    coord[c] = 2 * p[0] + (ch & 1);
    coord[(size_t)nc + c] = 2 * p[1] + ((ch >> 1) & 1);
    coord[(size_t)2 * nc + c] = d == 3 ? 2 * p[2] + ((ch >> 2) & 1) : 0;
    node_children[(size_t)node * nch + ch] = c;
  }
}

// neighbour of every cell side: a cell index, -1 on a transmissive boundary,
// -(node + 2) for a finer node across the side of a coarse cell; face counts:
// region 1 [dim][nc] conforming and boundary entries, region 2 [dim][nc][2]
// sub-face entries of coarse sides
__global__ void regrid_nbr_kernel(const BaseGrid g, const int32_t* __restrict__ first, const int32_t* __restrict__ node_of,
                           int nc, const int8_t* __restrict__ level, const int32_t* __restrict__ coord,
                           int32_t* __restrict__ nbr, uint8_t* __restrict__ scoarse, int32_t* __restrict__ cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int d = g.dim, l = level[c];
  const int nsub = 1 << (d - 1);
  const int pc[3] = {coord[c], coord[(size_t)nc + c], coord[(size_t)2 * nc + c]};
  unsigned coarse = 0;
  for (int a = 0; a < d; ++a)
    for (int s = 0; s < 2; ++s) {
      int p[3] = {pc[0], pc[1], pc[2]};
      p[a] += s ? 1 : -1;
      const int ext = g.n[a] << l;
      int32_t v;
      if ((p[a] < 0 || p[a] >= ext) && !g.periodic[a]) {
        v = -1;
      } else {
        p[a] = (p[a] + ext) % ext;
        const int b = (p[0] >> l) + g.n[0] * ((p[1] >> l) + g.n[1] * (p[2] >> l));
        const int nd = node_of[b];
        if (l == 0) v = nd >= 0 ? -(nd + 2) : first[b];
        else v = nd >= 0 ? first[b] + ((p[0] & 1) | ((p[1] & 1) << 1) | ((p[2] & 1) << 2)) : first[b];
      }
      nbr[(size_t)(2 * a + s) * nc + c] = v;
      if (v <= -2) coarse |= 1u << (2 * a + s);
      cnt[(size_t)d * nc + ((size_t)a * nc + c) * 2 + s] = v <= -2 ? nsub : 0;
    }
  scoarse[c] = (uint8_t)coarse;
  for (int a = 0; a < d; ++a) {
    const int up = nbr[(size_t)(2 * a + 1) * nc + c];
    const int dn = nbr[(size_t)(2 * a) * nc + c];
    cnt[(size_t)a * nc + c] = (up == -1) + (up >= 0 && level[up] == l) + (dn == -1);
  }
}

__global__ void regrid_faces_kernel(const BaseGrid g, int nc, const int8_t* __restrict__ level,
                             const int32_t* __restrict__ nbr, const int32_t* __restrict__ node_children,
                             const int32_t* __restrict__ off, int32_t* __restrict__ fm, int32_t* __restrict__ fp,
                             uint8_t* __restrict__ finfo, int32_t* __restrict__ sface) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = g.dim, nch = 1 << d, nsub = 1 << (d - 1);
  if (i >= (int64_t)d * nc) return;
  const int a = (int)(i / nc), c = (int)(i % nc);
  const int up = nbr[(size_t)(2 * a + 1) * nc + c];
  const int dn = nbr[(size_t)(2 * a) * nc + c];
  int f = off[i];
  if (up == -1) {
    fm[f] = c; fp[f] = -1; finfo[f] = (uint8_t)a;
    sface[(size_t)(2 * a + 1) * nc + c] = f++;
  } else if (up >= 0 && level[up] == level[c]) {
    fm[f] = c; fp[f] = up; finfo[f] = (uint8_t)a;
    sface[(size_t)(2 * a + 1) * nc + c] = f;
    sface[(size_t)(2 * a) * nc + up] = f++;
  }
  if (dn == -1) {
    fm[f] = -1; fp[f] = c; finfo[f] = (uint8_t)a;
    sface[(size_t)(2 * a) * nc + c] = f;
  }
  for (int s = 0; s < 2; ++s) {
    const int nb = s ? up : dn;
    if (nb > -2) continue;
    const int node = -(nb + 2);
    const int f0 = off[(size_t)d * nc + (size_t)i * 2 + s];
    for (int quad = 0; quad < nsub; ++quad) {
      // the child of the node in the layer next to the face, quadrant quad
      int ch = s ? 0 : (1 << a), t = 0;
      for (int b = 0; b < d; ++b) {
        if (b == a) continue;
        if ((quad >> t) & 1) ch |= 1 << b;
        ++t;
      }
      const int fine = node_children[(size_t)node * nch + ch];
      const int e = f0 + quad;
      if (s) { fm[e] = c; fp[e] = fine; finfo[e] = (uint8_t)(a | ((1 + quad) << 2)); }
      else { fm[e] = fine; fp[e] = c; finfo[e] = (uint8_t)(a | ((1 + quad) << 5)); }
      if (quad == 0) sface[(size_t)(2 * a + s) * nc + c] = e;
      sface[(size_t)(2 * a + 1 - s) * nc + fine] = e;
    }
  }
}

// one thread per output weight W_new[v][j][c]: blockIdx.y = v * N + j, cells along x
template <typename real>
__global__ void adapt_project_kernel(const BaseGrid g, int N, const double* __restrict__ P,
                               const int32_t* __restrict__ first0, const int32_t* __restrict__ node0,
                               const real* __restrict__ Wold, int nc0, const int8_t* __restrict__ level1,
                               const int32_t* __restrict__ coord1, int nc1, real* __restrict__ Wnew) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc1) return;
  const int vj = blockIdx.y;
  const int v = vj / N, j = vj % N;
  const size_t idx = (size_t)vj * nc1 + c;
  const int d = g.dim, nch = 1 << d;
  const int l = level1[c];
  const int p[3] = {coord1[c], coord1[(size_t)nc1 + c], coord1[(size_t)2 * nc1 + c]};
  const int b = (p[0] >> l) + g.n[0] * ((p[1] >> l) + g.n[1] * (p[2] >> l));
  const int ch = l ? ((p[0] & 1) | ((p[1] & 1) << 1) | ((p[2] & 1) << 2)) : 0;
  const int f0 = first0[b];
  const bool was_refined = node0[b] >= 0;
  const real* wv = Wold + (size_t)v * N * nc0;
  double val;
  if (was_refined == (l == 1)) {
    val = (double)wv[(size_t)j * nc0 + f0 + ch];
  } else if (l == 1) {  // w^c_j = sum_l P_c[j][l] w_l
    double s = 0.0;
    for (int m = 0; m < N; ++m)
      s = __dadd_rn(s, __dmul_rn(P[((size_t)ch * N + j) * N + m], (double)wv[(size_t)m * nc0 + f0]));
    val = s;
  } else {  // w_j = 2^-d sum_c sum_l P_c[l][j] w^c_l
    double s = 0.0;
    for (int cc = 0; cc < nch; ++cc)
      for (int m = 0; m < N; ++m)
        s = __dadd_rn(s, __dmul_rn(P[((size_t)cc * N + m) * N + j], (double)wv[(size_t)m * nc0 + f0 + cc]));
    val = scalbn(s, -d);
  }
  Wnew[idx] = (real)val;
}

}  // namespace

cudaError_t launch_adapt_criterion(const BaseGrid& g, const void* W, int esize, int N, int ncells,
                                   const int32_t* first, const int32_t* node_of, const double* P,
                                   double thr_leaf, double thr_node, uint8_t* crit, cudaStream_t s) {
  if (g.nbase == 0) return cudaSuccess;
  if (esize == 8)
    adapt_criterion_kernel<double><<<grid_for(g.nbase), RG_THREADS, 0, s>>>(
        g, static_cast<const double*>(W), N, ncells, first, node_of, P, thr_leaf, thr_node, crit);
  else
    adapt_criterion_kernel<float><<<grid_for(g.nbase), RG_THREADS, 0, s>>>(
        g, static_cast<const float*>(W), N, ncells, first, node_of, P, thr_leaf, thr_node, crit);
  return cudaGetLastError();
}

cudaError_t launch_adapt_buffer(const BaseGrid& g, const uint8_t* crit, const int32_t* node_of,
                                uint8_t* refined, int32_t* cnt, int32_t* changed, cudaStream_t s) {
  if (g.nbase == 0) return cudaSuccess;
  adapt_buffer_kernel<<<grid_for(g.nbase), RG_THREADS, 0, s>>>(g, crit, node_of, refined, cnt, changed);
  return cudaGetLastError();
}

cudaError_t launch_adapt_counts(const BaseGrid& g, const uint8_t* refined, const int32_t* node_of,
                                int32_t* cnt, int32_t* changed, cudaStream_t s) {
  if (g.nbase == 0) return cudaSuccess;
  adapt_counts_kernel<<<grid_for(g.nbase), RG_THREADS, 0, s>>>(g, refined, node_of, cnt, changed);
  return cudaGetLastError();
}

size_t scan_work_ints(int64_t n) { return (size_t)((n + SC_B - 1) / SC_B) + 1; }

cudaError_t launch_scan(const int32_t* in, int64_t n, int32_t* out, int32_t* work, cudaStream_t s) {
  const int nb = (int)((n + SC_B - 1) / SC_B);
  if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  regrid_scan_reduce_kernel<<<nb, SC_T, 0, s>>>(in, n, work);
  regrid_scan_blocks_kernel<<<1, SC_T, 0, s>>>(work, nb, out + n);
  regrid_scan_down_kernel<<<nb, SC_T, 0, s>>>(in, n, work, out);
  return cudaGetLastError();
}

cudaError_t launch_regrid_cells(const BaseGrid& g, const int32_t* first, int32_t* node_of, int ncells,
                                int8_t* level, int32_t* coord, int32_t* node_children, cudaStream_t s) {
  if (g.nbase == 0) return cudaSuccess;
  regrid_cells_kernel<<<grid_for(g.nbase), RG_THREADS, 0, s>>>(g, first, node_of, ncells, level, coord, node_children);
  return cudaGetLastError();
}

cudaError_t launch_regrid_nbr(const BaseGrid& g, const int32_t* first, const int32_t* node_of, int ncells,
                              const int8_t* level, const int32_t* coord, int32_t* nbr, uint8_t* scoarse,
                              int32_t* face_cnt, cudaStream_t s) {
  if (ncells == 0) return cudaSuccess;
  regrid_nbr_kernel<<<grid_for(ncells), RG_THREADS, 0, s>>>(g, first, node_of, ncells, level, coord, nbr, scoarse,
                                                      face_cnt);
  return cudaGetLastError();
}

cudaError_t launch_regrid_faces(const BaseGrid& g, int ncells, const int8_t* level, const int32_t* nbr,
                                const int32_t* node_children, const int32_t* face_off, int32_t* fm,
                                int32_t* fp, uint8_t* finfo, int32_t* sface, cudaStream_t s) {
  const int64_t n = (int64_t)g.dim * ncells;
  if (n == 0) return cudaSuccess;
  regrid_faces_kernel<<<grid_for(n), RG_THREADS, 0, s>>>(g, ncells, level, nbr, node_children, face_off, fm, fp,
                                                   finfo, sface);
  return cudaGetLastError();
}

cudaError_t launch_adapt_project(const BaseGrid& g, int esize, int nv, int N, const double* P,
                                 const int32_t* first0, const int32_t* node0, const void* Wold, int ncells0,
                                 const int8_t* level1, const int32_t* coord1, int ncells1, void* Wnew,
                                 cudaStream_t s) {
  if (ncells1 == 0) return cudaSuccess;
  const dim3 grid(grid_for(ncells1), nv * N);
  if (esize == 8)
    adapt_project_kernel<double><<<grid, RG_THREADS, 0, s>>>(g, N, P, first0, node0, static_cast<const double*>(Wold),
                                                       ncells0, level1, coord1, ncells1,
                                                       static_cast<double*>(Wnew));
  else
    adapt_project_kernel<float><<<grid, RG_THREADS, 0, s>>>(g, N, P, first0, node0, static_cast<const float*>(Wold),
                                                      ncells0, level1, coord1, ncells1,
                                                      static_cast<float*>(Wnew));
  return cudaGetLastError();
}

}  // namespace dgi
