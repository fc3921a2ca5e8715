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
  static __device__ __forceinline__ void lds(unsigned sa, A (&x)[V]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]) : "r"(sa));
  }
};

template <> struct Tr<__nv_bfloat16> {
  static constexpr int V = 4;
  using A = float;
  static __device__ __forceinline__ void unpack(const uint2 v, A (&x)[V]) {
    x[0] = __uint_as_float(v.x << 16);
    x[1] = __uint_as_float(v.x & 0xffff0000u);
    x[2] = __uint_as_float(v.y << 16);
    x[3] = __uint_as_float(v.y & 0xffff0000u);
  }
  static __device__ __forceinline__ void ld(const __nv_bfloat16* p, A (&x)[V]) {
    unpack(*reinterpret_cast<const uint2*>(p), x);
  }
  static __device__ __forceinline__ void ld_stream(const __nv_bfloat16* p, A (&x)[V]) {
    unpack(__ldcs(reinterpret_cast<const uint2*>(p)), x);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const A (&x)[V]) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]);  // round to nearest even
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(x[2], x[3]);
    __stcs(reinterpret_cast<uint2*>(p),
           make_uint2(*reinterpret_cast<const unsigned*>(&h0), *reinterpret_cast<const unsigned*>(&h1)));
  }
  static __device__ __forceinline__ double to_double(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
  static __device__ __forceinline__ void lds(unsigned sa, A (&x)[V]) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(sa));
    unpack(v, x);
  }
};

// Four floats from a 32-bit shared-memory address.
__device__ __forceinline__ void lds_f4(unsigned sa, float (&x)[4]) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]) : "r"(sa));
}

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
