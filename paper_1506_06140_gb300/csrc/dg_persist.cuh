// Whole RK steps in one persistent, cooperatively launched kernel (2D,
// states in FP64 or FP32, no gravity source): the phases of a step -- the
// CFL timestep (eq. time_step), and per stage the face fluxes, the cell
// update and, where the stage program asks for it, the slope and positivity
// limiters (Secs. 2.4, 3, 4.5) -- run back to back, separated by a grid-wide
// barrier instead of kernel launches.  On small meshes a step of the graph
// path is bound by the gaps between its launches; here a phase boundary
// costs one barrier.
//
// Each phase runs the same block bodies as the separate kernels (face,
// cell, limiter, positivity and timestep kernels), over virtual block
// indices strided by the grid, so results are bit for bit those of the
// launch-by-launch path with the default tiles (32 faces, 32 cells per
// block).  The arguments of every phase come from a plan in device memory,
// copied into shared memory once per launch.
//
// The barrier is a counter and a generation word in device memory (zeroed
// before each launch), with release/acquire atomics; its spin-wait gives up
// after a bounded number of polls (2^26), sets the abort word and the
// timeout status bit, and every block then leaves at its next barrier.  The cooperative launch guarantees that
// all blocks are resident at once (or fails to launch).
#pragma once
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_stage.cuh"

namespace dgi {

constexpr int PERSIST_THREADS = 128;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned x) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
  return old;
}

// bar[0] arrivals, bar[1] generation, bar[2] abort.  Returns false when the
// kernel must stop (a wait gave up here or elsewhere).  The block's writes
// are ordered before its arrival by the barrier and the release of the
// arrival; the acquire of the generation orders the other blocks' writes
// before the block's later reads.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblk, int* status) {
  __shared__ int pass;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = ld_acquire(&bar[2]) == 0u;
    if (ok) {
      const unsigned gen = ld_acquire(&bar[1]);
      if (atom_add_acq_rel(&bar[0], 1u) == nblk - 1u) {
        atomicExch(&bar[0], 0u);
        atom_add_acq_rel(&bar[1], 1u);
      } else {
        int it = 0;
        unsigned g;
        while ((g = ld_acquire(&bar[1])) == gen) {
          if ((++it & 1023) == 0) {
            if (ld_acquire(&bar[2]) != 0u) break;
            if (it > (1 << 26)) {
              atomicExch(&bar[2], 1u);
              atomicOr(status, 1 << DG_ERR_TIMEOUT_BIT);
              break;
            }
          }
        }
        ok = g != gen;
      }
    }
    pass = ok;
  }
  __syncthreads();
  return pass != 0;
}

template <typename real, int DIM, int K>
__global__ void __launch_bounds__(PERSIST_THREADS)
    persistent_steps_kernel(const PersistPlan<real>* plan, int n_steps, unsigned* bar, int* status) {
  static_assert(32 * Shape<DIM, K>::NV == PERSIST_THREADS, "2D: 32 faces or cells per block");
  static_assert(sizeof(PersistPlan<real>) % 16 == 0, "16-byte chunks");
  // the whole plan in shared memory, copied once per launch
  __shared__ __align__(16) unsigned char plan_sm[sizeof(PersistPlan<real>)];
  {
    const int4* s4 = reinterpret_cast<const int4*>(plan);
    int4* d4 = reinterpret_cast<int4*>(plan_sm);
    for (int i = threadIdx.x; i < (int)(sizeof(PersistPlan<real>) / 16); i += PERSIST_THREADS) d4[i] = s4[i];
  }
  PersistPlan<real>& P = *reinterpret_cast<PersistPlan<real>*>(plan_sm);
  double* const hist0 = plan->dt.dt_copy;
  __syncthreads();
  const unsigned nblk = gridDim.x;
  const int n_ops = P.n_ops;
  for (int step = 0; step < n_steps; ++step) {
    // timestep of the step (its last block writes dt and the history entry)
    if (threadIdx.x == 0 && hist0) P.dt.dt_copy = hist0 + (size_t)step * P.dt.m.nprob;
    __syncthreads();
    const int nd = P.dt_blocks;
    for (int b = blockIdx.x; b < nd; b += nblk) dt_body<real, DIM, K, PERSIST_THREADS>(P.dt, b, nd);
    if (!grid_barrier(bar, nblk, status)) return;
    for (int o = 0; o < n_ops; ++o) {
      const PersistOp<real>& op = P.op[o];
      for (int b = blockIdx.x; b < P.face_blocks; b += nblk) face_flux_body<real, DIM, K, 32>(op.st, b);
      if (!grid_barrier(bar, nblk, status)) return;
      for (int b = blockIdx.x; b < P.cell_blocks; b += nblk) cell_update_body<real, DIM, K, 32, false>(op.st, b);
      // the limiter's queue starts empty (its previous reader finished before the last barrier)
      if (op.lim && blockIdx.x == 0 && threadIdx.x == 0) *op.la.queue_len = 0;
      if (!grid_barrier(bar, nblk, status)) return;
      if (op.lim) {
        for (int b = blockIdx.x; b < P.lim_blocks; b += nblk) limit_body<real, DIM, K>(op.la, b);
        if (!grid_barrier(bar, nblk, status)) return;
        if (op.la.positivity && K > 0) {
          const int np = P.pos_blocks;
          for (int b = blockIdx.x; b < np; b += nblk) positivity_body<real, DIM, K>(op.la, b, np);
          if (!grid_barrier(bar, nblk, status)) return;
        }
      }
    }
  }
}

// dynamic shared memory of the persistent kernel: the larger of the face and
// cell bodies' tiles
template <typename real, int DIM, int K>
constexpr size_t persist_smem() {
  return FaceTile<real, DIM, K>::smem(32) > CellTile<real, DIM, K>::smem(32) ? FaceTile<real, DIM, K>::smem(32)
                                                                              : CellTile<real, DIM, K>::smem(32);
}

template <typename real, int DIM, int K>
struct PersistGrid {
  static inline int ctas = 0;  // co-resident blocks on the device (set by prepare_persist)
};

template <typename real, int DIM, int K>
cudaError_t prepare_persist() {
  auto f = persistent_steps_kernel<real, DIM, K>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)persist_smem<real, DIM, K>());
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, PERSIST_THREADS,
                                                         persist_smem<real, DIM, K>())) != cudaSuccess)
    return e;
  PersistGrid<real, DIM, K>::ctas = sms * per_sm;
  return cudaSuccess;
}

// blocks: the largest phase's virtual block count, at most the co-resident count
template <typename real, int DIM, int K>
cudaError_t launch_persist(const void* plan_dev, int max_phase_blocks, int n_steps, unsigned* bar, int* status,
                           cudaStream_t s) {
  const int cap = PersistGrid<real, DIM, K>::ctas;
  if (cap <= 0) return cudaErrorNotReady;
  int grid = max_phase_blocks < cap ? max_phase_blocks : cap;
  if (grid < 1) grid = 1;
  const PersistPlan<real>* p = static_cast<const PersistPlan<real>*>(plan_dev);
  void* args[] = {(void*)&p, (void*)&n_steps, (void*)&bar, (void*)&status};
  return cudaLaunchCooperativeKernel((const void*)persistent_steps_kernel<real, DIM, K>, dim3(grid),
                                     dim3(PERSIST_THREADS), args, persist_smem<real, DIM, K>(), s);
}

}  // namespace dgi
