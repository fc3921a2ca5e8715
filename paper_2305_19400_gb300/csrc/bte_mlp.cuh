// bte_mlp.cuh -- the learned temperature / equilibrium guess (device side).
//
// Two small networks with FP32 weights, 1 -> 64 -> 64 -> k, tanh hidden layers:
//   net A: normalised E_p -> normalised T (k = 1);
//   net B: normalised T   -> normalised I0_b(T)/I0_b(T_ref) for every band (k = nb).
// Parameter layout of one net: W1[64], b1[64], W2[64][64] (row o, column i),
// b2[64], W3[k][64], b3[k].  Inputs and outputs are affinely mapped to [-1, 1]
// over the training range.  A warp evaluates a net for one scalar input, with
// the forward-mode derivative of the outputs with respect to the input (for
// the surrogate Newton step on net B).
#pragma once
#include "bte_internal.h"

namespace bte {

constexpr int kHidden = 64;

__host__ __device__ inline int mlp_param_count(int k) { return 3 * kHidden + kHidden * kHidden + k * kHidden + k; }

struct MLPView {
  const float* A;         // net A parameters
  const float* B;         // net B parameters
  int nb;                 // outputs of net B
  double T_lo, T_hi;      // training temperature range
  double E_lo, E_hi;      // E_p(T_lo), E_p(T_hi)
  const double* r_lo;     // [nb] I0_b(T_lo)/I0_b(T_ref)
  const double* r_hi;     // [nb] I0_b(T_hi)/I0_b(T_ref)
  const double* I0ref;    // [nb] I0_b(T_ref)
};

// One warp: y[o] (and dy[o] = d y[o] / d x when dy != nullptr) for o < k into
// the warp's shared buffers.  h: 4 * kHidden floats of warp-private scratch.
__device__ inline void mlp_warp_eval(const float* __restrict__ p, int k, float x, float* y, float* dy, float* h) {
  const int lane = threadIdx.x & 31;
  const float* W1 = p;
  const float* b1 = W1 + kHidden;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + k * kHidden;
  float* h1 = h;
  float* d1 = h + kHidden;
  float* h2 = h + 2 * kHidden;
  float* d2 = h + 3 * kHidden;
  for (int u = lane; u < kHidden; u += 32) {
    const float t = tanhf(fmaf(W1[u], x, b1[u]));
    h1[u] = t;
    d1[u] = (1.f - t * t) * W1[u];
  }
  __syncwarp();
  for (int u = lane; u < kHidden; u += 32) {
    float z = b2[u], dz = 0.f;
    for (int i = 0; i < kHidden; ++i) {
      z = fmaf(W2[u * kHidden + i], h1[i], z);
      dz = fmaf(W2[u * kHidden + i], d1[i], dz);
    }
    const float t = tanhf(z);
    h2[u] = t;
    d2[u] = (1.f - t * t) * dz;
  }
  __syncwarp();
  for (int o = lane; o < k; o += 32) {
    float z = b3[o], dz = 0.f;
    for (int j = 0; j < kHidden; ++j) {
      z = fmaf(W3[o * kHidden + j], h2[j], z);
      dz = fmaf(W3[o * kHidden + j], d2[j], dz);
    }
    y[o] = z;
    if (dy) dy[o] = dz;
  }
  __syncwarp();
}

// Learned start of the T_p solve for one cell (whole warp): net A's guess from
// E_p, then `nsur` Newton steps on the surrogate residual
//   F~(T) = sum_b a_p,b I0ref_b r_b(T) - E_p,  r_b from net B.
// ybuf: 2 * nb floats, h: 4 * kHidden floats (warp-private shared memory).
__device__ inline double mlp_guess_T(const MLPView& m, const double* a_p, double Ep, int nsur, float* ybuf, float* h) {
  const int lane = threadIdx.x & 31;
  const double span = m.T_hi - m.T_lo;
  const float xe = (float)(2.0 * (Ep - m.E_lo) / (m.E_hi - m.E_lo) - 1.0);
  mlp_warp_eval(m.A, 1, xe, ybuf, nullptr, h);
  double T = m.T_lo + 0.5 * ((double)ybuf[0] + 1.0) * span;
  for (int it = 0; it < nsur; ++it) {
    const float xt = (float)(2.0 * (T - m.T_lo) / span - 1.0);
    mlp_warp_eval(m.B, m.nb, xt, ybuf, ybuf + m.nb, h);
    double F = 0.0, dF = 0.0;
    for (int b = lane; b < m.nb; b += 32) {
      const double half = 0.5 * (m.r_hi[b] - m.r_lo[b]);
      const double w = a_p[b] * m.I0ref[b];
      F = fma(w, m.r_lo[b] + half * ((double)ybuf[b] + 1.0), F);
      dF = fma(w, half * (double)ybuf[m.nb + b] * (2.0 / span), dF);
    }
    for (int o = 16; o > 0; o >>= 1) {
      F += __shfl_xor_sync(0xffffffffu, F, o);
      dF += __shfl_xor_sync(0xffffffffu, dF, o);
    }
    F -= Ep;
    if (!(dF > 0.0) || !isfinite(F)) break;
    const double Tn = T - F / dF;
    if (!(Tn >= kTmin && Tn <= kTmax)) break;
    T = Tn;
  }
  return T;
}

}  // namespace bte
