// bte_sweep_fp32.cu -- sweep kernel instances for FP32 intensity storage.
#include "bte_sweep.cuh"

namespace bte {

cudaError_t launch_sweep_fp32(int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  return sweep::launch<float>(pd, a, dim, threads, grid, s);
}

}  // namespace bte
