// bte_sweep_fp64.cu -- sweep kernel instances for FP64 intensity storage.
#include "bte_sweep.cuh"
#include "bte_sweep_ff.cuh"

namespace bte {

cudaError_t launch_sweep_fp64(int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  if (a.ff != 0) return sweep_ff::launch(pd, a, dim, threads, grid, s);  // double-float arithmetic
  return sweep::launch<double>(pd, a, dim, threads, grid, s);
}

}  // namespace bte
