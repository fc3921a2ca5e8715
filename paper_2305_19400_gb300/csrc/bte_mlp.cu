// bte_mlp.cu -- training and batch-inference kernels of the learned guess.
//
// Training pairs come from the library's own FP64 band quadrature: for a
// counter-based uniform T in [T_lo, T_hi], I0_b(T) for every band and
// E_p(T) = sum_b a_p,b I0_b(T).  Net A learns E_p -> T, net B learns
// T -> I0_b(T)/I0_b(T_ref).  Activations are stored [feature][sample] with the
// sample index fastest; every reduction over a minibatch is done by one thread
// in a fixed order, so training is deterministic.
#include <algorithm>

#include "bte_mlp.cuh"
#include "bte_quad.cuh"
#include "bte_solve.cuh"

namespace bte {

namespace {

// SplitMix64 finaliser of (seed, counter) -> uniform double in [0, 1).
__device__ __forceinline__ double counter_uniform(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Reference values: I0_b at T_lo, T_hi, T_ref -> r_lo, r_hi (ratios), E_lo, E_hi.
__global__ void mlp_norm_kernel(ThermoTables th, double T_lo, double T_hi, const double* I0ref, double* r_lo,
                                double* r_hi, double* E_lohi) {
  __shared__ double s_lo[256], s_hi[256];
  const int b = threadIdx.x;
  double elo = 0.0, ehi = 0.0;
  if (b < th.nb) {
    const double flo = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, 1.0 / T_lo);
    const double fhi = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, 1.0 / T_hi);
    r_lo[b] = flo / I0ref[b];
    r_hi[b] = fhi / I0ref[b];
    elo = th.a_p[b] * flo;
    ehi = th.a_p[b] * fhi;
  }
  s_lo[b] = elo;
  s_hi[b] = ehi;
  __syncthreads();
  if (b == 0) {
    double a = 0.0, c = 0.0;
    for (int i = 0; i < th.nb; ++i) { a += s_lo[i]; c += s_hi[i]; }
    E_lohi[0] = a;
    E_lohi[1] = c;
  }
}

// One training pair per thread.  xA = normalised E_p, yA = xB = normalised T,
// yB[b][n] = normalised I0_b/I0_b(T_ref).
__global__ void mlp_pairs_kernel(ThermoTables th, double T_lo, double T_hi, const double* I0ref, const double* r_lo,
                                 const double* r_hi, const double* E_lohi, unsigned long long seed, int n, float* xA,
                                 float* yA, float* yB) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double T = T_lo + (T_hi - T_lo) * counter_uniform(seed, (unsigned long long)i);
    const double rT = 1.0 / T;
    double Ep = 0.0;
    for (int b = 0; b < th.nb; ++b) {
      const double f = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, rT);
      Ep = fma(th.a_p[b], f, Ep);
      yB[(size_t)b * n + i] = (float)(2.0 * (f / I0ref[b] - r_lo[b]) / (r_hi[b] - r_lo[b]) - 1.0);
    }
    xA[i] = (float)(2.0 * (Ep - E_lohi[0]) / (E_lohi[1] - E_lohi[0]) - 1.0);
    yA[i] = (float)(2.0 * (T - T_lo) / (T_hi - T_lo) - 1.0);
  }
}

// H[o][n] = act(b[o] + sum_i W[o][i] X[i][n]), X with leading dimension ldx.
__global__ void dense_fwd_kernel(const float* W, const float* b, const float* X, int ldx, float* H, int out, int in,
                                 int B, int act) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= out * B) return;
  const int o = idx / B, n = idx - o * B;
  float z = b[o];
  for (int i = 0; i < in; ++i) z = fmaf(W[o * in + i], X[(size_t)i * ldx + n], z);
  H[idx] = act ? tanhf(z) : z;
}

// dY = 2 (Y - Tg) / (k B) and per-block partial sums of (Y - Tg)^2 / (k B).
__global__ void mse_kernel(const float* Y, const float* Tg, int ldt, float* dY, float* part, int k, int B) {
  __shared__ float sh[256];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (idx < k * B) {
    const int o = idx / B, n = idx - o * B;
    const float e = Y[idx] - Tg[(size_t)o * ldt + n];
    dY[idx] = 2.f * e / (float)(k * B);
    l = e * e / (float)(k * B);
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) sh[threadIdx.x] += sh[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// dW[o][i] = sum_n dZ[o][n] X[i][n]; db[o] = sum_n dZ[o][n] (threads over o*(in+1)).
__global__ void dense_bwd_w_kernel(const float* dZ, const float* X, int ldx, float* dW, float* db, int out, int in,
                                   int B) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= out * (in + 1)) return;
  const int o = idx / (in + 1), i = idx - o * (in + 1);
  float acc = 0.f;
  if (i < in) {
    for (int n = 0; n < B; ++n) acc = fmaf(dZ[(size_t)o * B + n], X[(size_t)i * ldx + n], acc);
    dW[o * in + i] = acc;
  } else {
    for (int n = 0; n < B; ++n) acc += dZ[(size_t)o * B + n];
    db[o] = acc;
  }
}

// dZp[i][n] = (sum_o W[o][i] dZ[o][n]) (1 - Hp[i][n]^2)   (back through a tanh layer)
__global__ void dense_bwd_x_kernel(const float* W, const float* dZ, const float* Hp, float* dZp, int out, int in, int B) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= in * B) return;
  const int i = idx / B, n = idx - i * B;
  float acc = 0.f;
  for (int o = 0; o < out; ++o) acc = fmaf(W[o * in + i], dZ[(size_t)o * B + n], acc);
  const float h = Hp[idx];
  dZp[idx] = acc * (1.f - h * h);
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Batch solve of the T_p equation for energies Ep[i] (one warp each): optional
// learned start, then the exact solve.  Writes T and the evaluation count.
__global__ void solve_batch_kernel(ThermoTables th, const double* Ep, const double* T0, int n, double trust_rel,
                                   int maxit, int learned, MLPView m, double* Tout, int* evals) {
  extern __shared__ float fsm[];
  const int warps = blockDim.x / 32, lane = threadIdx.x & 31, wid = threadIdx.x / 32;
  float* ybuf = fsm + (size_t)wid * (2 * th.nbp + 4 * kHidden);
  float* hbuf = ybuf + 2 * th.nbp;
  for (int w = blockIdx.x * warps + wid; w < n; w += gridDim.x * warps) {
    const double start = learned ? mlp_guess_T(m, th.a_p, Ep[w], 2, ybuf, hbuf) : (T0 ? T0[w] : 300.0);
    const SolveResult r = exact_solve_warp(th, Ep[w], start, trust_rel, maxit, nullptr);
    if (lane == 0) {
      Tout[w] = r.bad ? NAN : r.Te + r.delta;
      evals[w] = r.evals;
    }
  }
}

inline int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int mlp_param_total(int nb) { return mlp_param_count(1) + mlp_param_count(nb); }

cudaError_t launch_mlp_norm(ThermoTables th, double T_lo, double T_hi, const double* I0ref, double* r_lo, double* r_hi,
                            double* E_lohi, cudaStream_t s) {
  mlp_norm_kernel<<<1, 256, 0, s>>>(th, T_lo, T_hi, I0ref, r_lo, r_hi, E_lohi);
  return cudaGetLastError();
}

cudaError_t launch_mlp_pairs(ThermoTables th, double T_lo, double T_hi, const double* I0ref, const double* r_lo,
                             const double* r_hi, const double* E_lohi, unsigned long long seed, int n, float* xA,
                             float* yA, float* yB, cudaStream_t s) {
  mlp_pairs_kernel<<<std::min(blocks(n, 128), 152 * 32), 128, 0, s>>>(th, T_lo, T_hi, I0ref, r_lo, r_hi, E_lohi, seed, n,
                                                                       xA, yA, yB);
  return cudaGetLastError();
}

// One net: forward, MSE and backward over a minibatch of B samples starting at
// column `off` of the inputs X (ld ldx) and targets Tg (ld ldt).  grad has the
// parameter layout; act holds 4*64*B + 2*k*B floats of activations and
// gradients; part receives ceil(k*B/256) loss partials.
cudaError_t mlp_forward_backward(const float* p, int k, const float* X, int ldx, const float* Tg, int ldt, int B,
                                 float* grad, float* act, float* part, cudaStream_t s) {
  const float* W1 = p;
  const float* b1 = W1 + kHidden;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + k * kHidden;
  float* gW1 = grad;
  float* gb1 = gW1 + kHidden;
  float* gW2 = gb1 + kHidden;
  float* gb2 = gW2 + kHidden * kHidden;
  float* gW3 = gb2 + kHidden;
  float* gb3 = gW3 + k * kHidden;
  float* H1 = act;
  float* H2 = H1 + kHidden * B;
  float* dZ1 = H2 + kHidden * B;
  float* dZ2 = dZ1 + kHidden * B;
  float* Y = dZ2 + kHidden * B;
  float* dY = Y + k * B;
  const int t = 256;
  dense_fwd_kernel<<<blocks((long long)kHidden * B, t), t, 0, s>>>(W1, b1, X, ldx, H1, kHidden, 1, B, 1);
  dense_fwd_kernel<<<blocks((long long)kHidden * B, t), t, 0, s>>>(W2, b2, H1, B, H2, kHidden, kHidden, B, 1);
  dense_fwd_kernel<<<blocks((long long)k * B, t), t, 0, s>>>(W3, b3, H2, B, Y, k, kHidden, B, 0);
  mse_kernel<<<blocks((long long)k * B, t), t, 0, s>>>(Y, Tg, ldt, dY, part, k, B);
  dense_bwd_w_kernel<<<blocks((long long)k * (kHidden + 1), t), t, 0, s>>>(dY, H2, B, gW3, gb3, k, kHidden, B);
  dense_bwd_x_kernel<<<blocks((long long)kHidden * B, t), t, 0, s>>>(W3, dY, H2, dZ2, k, kHidden, B);
  dense_bwd_w_kernel<<<blocks((long long)kHidden * (kHidden + 1), t), t, 0, s>>>(dZ2, H1, B, gW2, gb2, kHidden, kHidden,
                                                                                  B);
  dense_bwd_x_kernel<<<blocks((long long)kHidden * B, t), t, 0, s>>>(W2, dZ2, H1, dZ1, kHidden, kHidden, B);
  dense_bwd_w_kernel<<<blocks((long long)kHidden * 2, t), t, 0, s>>>(dZ1, X, ldx, gW1, gb1, kHidden, 1, B);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<blocks(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_solve_batch(ThermoTables th, const double* Ep, const double* T0, int n, double trust_rel, int maxit,
                               const MLPView* mlp, double* Tout, int* evals, cudaStream_t s) {
  const size_t sm = 4 * (2 * (size_t)th.nbp + 4 * kHidden) * sizeof(float);
  MLPView m{};
  if (mlp) m = *mlp;
  solve_batch_kernel<<<std::min(blocks(n, 4), 152 * 8), 128, sm, s>>>(th, Ep, T0, n, trust_rel, maxit, mlp ? 1 : 0, m,
                                                                      Tout, evals);
  return cudaGetLastError();
}

}  // namespace bte
