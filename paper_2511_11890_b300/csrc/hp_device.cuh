// Device helpers for libhp kernels (sm_103a): mbarriers with bounded waits,
// TMA tile loads, element conversion.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hp_internal.h"

namespace hp {

// Poll limit of a bounded mbarrier wait. A try_wait on an incomplete phase
// suspends the thread for a few microseconds before it returns false
// (measured on B300: 2^22 polls took 16 s), so 2^18 polls give up after about
// one second, far above any TMA completion time of a healthy GPU.
constexpr uint32_t kWaitLimit = 1u << 18;

// Error word codes (OR-ed together).
constexpr int kErrTimeout = 1;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 3D TMA tile load (x, y, z coordinates, x innermost) into shared memory,
// completing on `bar` with the transferred byte count.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Element -> float. uint16 uses the exact 2^23 bias trick (one LOP + one
// FADD instead of an integer-to-float conversion).
template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<uint8_t>(uint8_t v) {
  return __int_as_float(0x4B000000 | (uint32_t)v) - 8388608.0f;
}
template <>
__device__ __forceinline__ float to_f32<uint16_t>(uint16_t v) {
  return __int_as_float(0x4B000000 | (uint32_t)v) - 8388608.0f;
}
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) {
  return __half2float(v);
}
template <>
__device__ __forceinline__ float to_f32<float>(float v) {
  return v;
}

template <typename T>
struct DtypeOf;
template <>
struct DtypeOf<uint8_t> {
  static constexpr int value = HP_U8;
};
template <>
struct DtypeOf<uint16_t> {
  static constexpr int value = HP_U16;
};
template <>
struct DtypeOf<__half> {
  static constexpr int value = HP_F16;
};
template <>
struct DtypeOf<float> {
  static constexpr int value = HP_F32;
};

// Packed FP32 pair arithmetic (Blackwell fma.rn.f32x2): one instruction,
// two independent IEEE fmas, each rounded exactly like fmaf.
__device__ __forceinline__ unsigned long long pack2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long splat2(float g) { return pack2(make_float2(g, g)); }

// Four consecutive elements -> float4 (vectorised staging of interior tiles).
template <typename T>
__device__ __forceinline__ float4 load4_f32(const T* p);
template <>
__device__ __forceinline__ float4 load4_f32<uint8_t>(const uint8_t* p) {
  const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
  return make_float4(to_f32<uint8_t>(v & 0xFF), to_f32<uint8_t>((v >> 8) & 0xFF),
                     to_f32<uint8_t>((v >> 16) & 0xFF), to_f32<uint8_t>(v >> 24));
}
template <>
__device__ __forceinline__ float4 load4_f32<uint16_t>(const uint16_t* p) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  return make_float4(to_f32<uint16_t>(v.x & 0xFFFF), to_f32<uint16_t>(v.x >> 16),
                     to_f32<uint16_t>(v.y & 0xFFFF), to_f32<uint16_t>(v.y >> 16));
}
template <>
__device__ __forceinline__ float4 load4_f32<__half>(const __half* p) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 load4_f32<float>(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

__device__ __forceinline__ void set_device_error(int* err, int code) {
  if (err) atomicOr(err, code);
}

}  // namespace hp
