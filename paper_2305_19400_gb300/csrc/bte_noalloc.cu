// bte_noalloc.cu -- wall heat flux without any device allocation.
//
// Some callers cannot call cudaMalloc: processes that run under a fixed
// device-memory budget or whose device memory is owned by another allocator
// (for example a framework's caching allocator that holds the whole GPU), and
// latency-critical loops in which cudaMalloc/cudaFree would synchronize the
// device.  bte_get_wall_flux_noalloc serves them: it computes the same
// per-side mean outgoing wall flux as bte_get_flux, but its per-face partial
// sums live in the file-scope device array below instead of in a workspace.
//
// The array is a static __device__ object, so every GPU that loads libbte.so
// holds it (kNoAllocMaxFaces + 8 doubles, 512 KB + 64 B) until the process
// exits.  In host code its name is only a host-side stand-in, never a device
// address: the device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <mutex>

#include "../../include/bte.h"
#include "bte_internal.h"

namespace bte {
namespace {

constexpr int kNoAllocMaxFaces = 65536;
constexpr int kNoAllocMaxDevices = 64;

// [0, kNoAllocMaxFaces): per-face sums of one wall; [kNoAllocMaxFaces, +6): per-side means.
static __device__ __align__(256) double g_wall_scratch[kNoAllocMaxFaces + 8];

std::mutex g_setup_mu;
double* g_scratch_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_wall_scratch on device `dev`, which must be current
// (set up on first use).
cudaError_t scratch_address(int dev, double** out) {
  cudaError_t e = cudaSuccess;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_wall_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__device__ double block_sum_static(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Net outgoing flux through each face of one wall; face sums go to scratch[f].
__global__ void wall_faces_static_kernel(const double* I, const double* I0wall, const DevGeom* geoms, int geom,
                                         int side, const DirInfo* dirs, const double* S, int nd, int nbp,
                                         double* scratch, int nfaces) {
  __shared__ double sh[256];
  const DevGeom g = geoms[geom];
  const int ax = side / 2;
  const double nsign = (side & 1) ? 1.0 : -1.0;
  const int bc = g.bc[side];
  const long long f0 = g.face0[side];
  for (int f = blockIdx.x; f < nfaces; f += gridDim.x) {
    int i, j, k;
    if (side < 2) { j = f % g.ny; k = f / g.ny; i = (side & 1) ? g.nx - 1 : 0; }
    else if (side < 4) { i = f % g.nx; k = f / g.nx; j = (side & 1) ? g.ny - 1 : 0; }
    else { i = f % g.nx; j = f / g.nx; k = (side & 1) ? g.nz - 1 : 0; }
    const long long P = g.cell0 + i + (long long)g.nx * (j + (long long)g.ny * k);
    const double* row = I + P * (long long)nd * nbp;
    double acc = 0.0;
    for (long long e = threadIdx.x; e < (long long)nd * nbp; e += blockDim.x) {
      const int d = (int)(e / nbp);
      const int b = (int)(e - (long long)d * nbp);
      const double sn = S[3 * d + ax] * nsign;
      double v;
      if (sn > 0.0) v = row[e];
      else if (bc == 0) v = I0wall[(f0 + f) * nbp + b];
      else if (bc == 3) v = reinterpret_cast<const double*>(g.gdir[side])[(long long)f * nd * nbp + e];
      else {
        const int r = ax == 0 ? dirs[d].rx : (ax == 1 ? dirs[d].ry : dirs[d].rz);
        v = row[(long long)r * nbp + b];
      }
      acc = fma(sn, v, acc);
    }
    const double t = block_sum_static(acc, sh);
    if (threadIdx.x == 0) scratch[f] = t;
  }
}

// Mean of scratch[0, n) into scratch[kNoAllocMaxFaces + side].
__global__ void wall_mean_static_kernel(double* scratch, int n, int side) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc += scratch[e];
  const double t = block_sum_static(acc, sh);
  if (threadIdx.x == 0) scratch[kNoAllocMaxFaces + side] = t / (double)n;
}

}  // namespace
}  // namespace bte

namespace bte {
namespace {
int wall_flux_on_device(bte_handle h, const FluxView& v, int geom, double* q_walls, int out_on_device);
}  // namespace
}  // namespace bte

using namespace bte;

extern "C" int bte_get_wall_flux_noalloc(bte_handle h, int geom, double* q_walls, int out_on_device) {
  if (!h) return BTE_E_ARG;
  if (!q_walls) return set_handle_error(h, BTE_E_ARG, "q_walls is NULL");
  // The handle's memory and stream, and the scratch address used here, belong
  // to the handle's device: make it current for the wall-ghost refresh, the
  // address lookup and the launches, and give the caller's device back.
  const int dev = handle_device(h);
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
  if (e != cudaSuccess) return set_handle_error(h, BTE_E_CUDA, "cudaSetDevice(%d): %s", dev, cudaGetErrorString(e));
  FluxView v;
  int rc = flux_view(h, geom, &v);
  if (rc == BTE_OK) {
    if (v.precision != BTE_FP64) {
      rc = set_handle_error(h, BTE_E_ARG, "the no-allocation wall flux serves FP64 handles only");
    } else {
      for (int side = 0; side < 2 * v.dim && rc == BTE_OK; ++side)
        if (v.nfaces[side] > kNoAllocMaxFaces)
          rc = set_handle_error(h, BTE_E_ARG, "wall %d has %d faces; the no-allocation path holds at most %d per wall",
                                side, v.nfaces[side], kNoAllocMaxFaces);
      if (rc == BTE_OK) rc = wall_flux_on_device(h, v, geom, q_walls, out_on_device);
    }
  }
  if (prev != dev) cudaSetDevice(prev);
  return rc;
}

namespace bte {
namespace {
int wall_flux_on_device(bte_handle h, const FluxView& v, int geom, double* q_walls, int out_on_device) {
  double* scratch = nullptr;
  cudaError_t e = scratch_address(v.dev, &scratch);
  if (e != cudaSuccess) return set_handle_error(h, BTE_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  for (int side = 0; side < 2 * v.dim; ++side) {
    const int nf = v.nfaces[side];
    const int grid = nf < 152 * 16 ? nf : 152 * 16;
    wall_faces_static_kernel<<<grid, 256, 0, v.stream>>>(v.I, v.I0wall, v.geoms, geom, side, v.dirs, v.S, v.nd,
                                                         v.nbp, scratch, nf);
    wall_mean_static_kernel<<<1, 256, 0, v.stream>>>(scratch, nf, side);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q_walls, scratch + kNoAllocMaxFaces, 2 * v.dim * sizeof(double),
                        out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) return set_handle_error(h, BTE_E_CUDA, "wall flux: %s", cudaGetErrorString(e));
  return BTE_OK;
}
}  // namespace
}  // namespace bte
