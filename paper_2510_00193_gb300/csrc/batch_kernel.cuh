// Batched energy/force/virial/gradient evaluation of many small periodic
// configurations in one persistent launch.
//
// Work items are (configuration, first atom, atom count) with count <= the
// block size (the tuned "atoms per block"); a block takes items from a
// global counter until none are left.  Each item's atoms belong to one
// configuration, so the block reduces energy, virial and dE/dtheta in shared
// memory and adds them to that configuration's slots with one FP64 atomic per
// value.  The per-atom work is the single-configuration code (efv_atom), with
// the whole-DAG contraction: inside the persistent loop the per-graph form
// spills more (1.5-1.8 KB against 0.7-0.9 KB per thread at level 16) and
// measured slower (1.80 against 1.76 ms for the 4096-configuration batch
// with dE/dtheta; the per-graph form in a non-inlined per-item function needs
// no stack but took 2.25 ms).
#pragma once
#include "efv_kernel.cuh"

namespace mtp {

struct BatchArgs {
  EfvArgs base;               // lists, positions, parameters, forces, status
  const int32_t* item_cfg;    // [n_items]
  const int64_t* item_begin;  // [n_items]
  const int32_t* item_count;  // [n_items]
  int32_t n_items;
  int32_t* queue;             // work counter, zero at launch
  const double* cells;        // [n_cfg][9]
  double* e_cfg;              // [n_cfg]
  double* virial_cfg;         // [n_cfg][6]
  double* dtheta_cfg;         // [n_cfg][n_params] or null
  int64_t n_params;
};

template <class LV, class R, bool DTHETA, int NQ = 0>
__global__ void __launch_bounds__(256) batch_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ R s_cell[9];
  const EfvArgs& a = b.base;
  EfvShared<R, LV::NMU, DTHETA> sm;
  sm.setup(a, smem_raw);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(b.queue, 1);
    sm.zero_gradients();
    __syncthreads();
    const int it = s_item;
    if (it >= b.n_items) break;
    const int cfg = b.item_cfg[it];
    const int64_t first = b.item_begin[it];
    const int count = b.item_count[it];
    if (threadIdx.x < 9) s_cell[threadIdx.x] = R(b.cells[(int64_t)cfg * 9 + threadIdx.x]);
    __syncthreads();
    double e_i = 0.0;
    R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const bool active = (int)threadIdx.x < count;
    if (__any_sync(0xffffffffu, active))   // warp-uniform: whole warps without atoms skip the work
      efv_atom<LV, R, DTHETA, false, NQ, true>(a, sm, active ? first + threadIdx.x : first, active, s_cell, nullptr,
                                               e_i, w);
    efv_block_flush<LV, R, DTHETA>(sm, e_i, w, b.e_cfg + cfg, b.virial_cfg + (int64_t)cfg * 6,
                                   DTHETA ? b.dtheta_cfg + (int64_t)cfg * b.n_params : nullptr);
    __syncthreads();
  }
}

template <class LV, class R, bool DTHETA>
int batch_launch_typed(const BatchArgs& b, int threads, cudaStream_t stream) {
  const int SS = b.base.n_species * b.base.n_species;
  const size_t bytes = ((efv_smem_bytes<R, LV::NMU, DTHETA>(SS, b.base.n_q, b.base.m) + 15) & ~size_t(15)) +
                       efv_acc_bytes<R, LV::NMU, DTHETA>(b.base.n_species, b.base.n_q, threads);
  auto kern = batch_kernel<LV, R, DTHETA>;
  if constexpr (std::is_same<R, float>::value && LV::NGROUPS == 1) {
    if (b.base.n_q == kFixedQ) kern = batch_kernel<LV, R, DTHETA, kFixedQ>;
  }
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
  }
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, bytes);
  const int grid = std::max(1, std::min(b.n_items, std::max(1, per_sm) * sms));
  kern<<<grid, threads, bytes, stream>>>(b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("batch kernel launch (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

template <class LV>
int batch_launch(const BatchArgs& b, int precision, bool want_dtheta, int threads, cudaStream_t stream) {
  if (precision == MTP_MIXED)
    return want_dtheta ? batch_launch_typed<LV, float, true>(b, threads, stream)
                       : batch_launch_typed<LV, float, false>(b, threads, stream);
  return want_dtheta ? batch_launch_typed<LV, double, true>(b, threads, stream)
                     : batch_launch_typed<LV, double, false>(b, threads, stream);
}

}  // namespace mtp
