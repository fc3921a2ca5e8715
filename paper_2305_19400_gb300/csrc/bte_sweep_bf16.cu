// bte_sweep_bf16.cu -- sweep kernel instances for BF16 intensity storage.
#include "bte_sweep.cuh"

namespace bte {

cudaError_t launch_sweep_bf16(int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  return sweep::launch<__nv_bfloat16>(pd, a, dim, threads, grid, s);
}

}  // namespace bte
