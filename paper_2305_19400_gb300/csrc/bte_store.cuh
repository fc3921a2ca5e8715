// bte_store.cuh -- storage traits of the intensity buffers (FP64 / FP32 / BF16)
// and small load helpers, shared by the library's kernels.
#pragma once
#include <cuda_bf16.h>

#include "bte_internal.h"

namespace bte {

// Storage traits: V values per vector load, arithmetic type A.
template <typename S> struct Tr;

template <> struct Tr<double> {
  static constexpr int V = 2;
  using A = double;
  static __device__ __forceinline__ void ld(const double* p, A (&x)[V]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
  static __device__ __forceinline__ void ld_stream(const double* p, A (&x)[V]) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
  }
  static __device__ __forceinline__ void st(double* p, const A (&x)[V]) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
  }
  static __device__ __forceinline__ double to_double(double v) { return v; }
  // V values from a 32-bit shared-memory address
  static __device__ __forceinline__ void lds(unsigned sa, A (&x)[V]) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x[0]), "=d"(x[1]) : "r"(sa));
  }
};

template <> struct Tr<float> {
  static constexpr int V = 4;
  using A = float;
  static __device__ __forceinline__ void ld(const float* p, A (&x)[V]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  static __device__ __forceinline__ void ld_stream(const float* p, A (&x)[V]) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const A (&x)[V]) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
  }
  static __device__ __forceinline__ double to_double(float v) { return (double)v; }
  static __device__ __forceinline__ float to_float(float v) { return v; }
  static __device__ __forceinline__ float from_float(float v) { return v; }
  static __device__ __forceinline__ void lds(unsigned sa, A (&x)[V]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]) : "r"(sa));
  }
};

// BF16: a lane holds 8 bands (one 16-byte vector), so the per-step overhead of
// the sweep is spread over as many updates as FP32 moves in 32 bytes.
template <> struct Tr<__nv_bfloat16> {
  static constexpr int V = 8;
  using A = float;
  static __device__ __forceinline__ void unpack(const uint4 v, A (&x)[V]) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[2 * i] = __uint_as_float(w[i] << 16);
      x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
  static __device__ __forceinline__ unsigned pack2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // round to nearest even
    return *reinterpret_cast<const unsigned*>(&h);
  }
  static __device__ __forceinline__ void ld(const __nv_bfloat16* p, A (&x)[V]) {
    unpack(*reinterpret_cast<const uint4*>(p), x);
  }
  static __device__ __forceinline__ void ld_stream(const __nv_bfloat16* p, A (&x)[V]) {
    unpack(__ldcs(reinterpret_cast<const uint4*>(p)), x);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const A (&x)[V]) {
    __stcs(reinterpret_cast<uint4*>(p),
           make_uint4(pack2(x[0], x[1]), pack2(x[2], x[3]), pack2(x[4], x[5]), pack2(x[6], x[7])));
  }
  static __device__ __forceinline__ double to_double(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
  static __device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 from_float(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ void lds(unsigned sa, A (&x)[V]) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(sa));
    unpack(v, x);
  }
};

// V consecutive values of type A from global memory (16-byte loads).
template <typename A, int V>
__device__ __forceinline__ void ldgv(const A* p, A (&x)[V]) {
  if constexpr (sizeof(A) == 8) {
#pragma unroll
    for (int i = 0; i < V; i += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(p + i));
      x[i] = v.x; x[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + i));
      x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
    }
  }
}

// Full intensity value (FP64) of element e of a padded row set (the reduced
// modes store the deviation from I0_b(T_ref)).
template <typename S>
__device__ __forceinline__ double full_I(const S* I, long long e, int b, const double* I0ref) {
  if constexpr (sizeof(S) == 8) return (double)I[e];
  else return I0ref[b] + Tr<S>::to_double(I[e]);
}

}  // namespace bte
