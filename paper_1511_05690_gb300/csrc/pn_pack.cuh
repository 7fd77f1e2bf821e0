// Conversion of powered operand values to the tensor-core operand formats:
// 16 bytes of an operand tile image from EPC values (BF16, FP16, E4M3, TF32,
// or the hi/lo TF32 pair of the 3xTF32 split).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "pn_device.cuh"

namespace pn {

// x^(2^plog) by repeated squaring (each step one correctly rounded multiply).
__device__ __forceinline__ float pow2k(float x, int plog) {
#pragma unroll 1
  for (int t = 0; t < plog; ++t) x = x * x;
  return x;
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Packs 16 bytes of operand data from EPC powered, shifted values.
template <int MODE>
struct Packer;

template <>
struct Packer<MODE_BF16> {
  static constexpr int EPC = 8;
  __device__ static void pack(const float (&v)[EPC], uint4& hi, uint4&) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    hi = make_uint4(w[0], w[1], w[2], w[3]);
  }
};

template <>
struct Packer<MODE_F16> {
  static constexpr int EPC = 8;
  __device__ static void pack(const float (&v)[EPC], uint4& hi, uint4&) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    hi = make_uint4(w[0], w[1], w[2], w[3]);
  }
};

template <>
struct Packer<MODE_E4M3> {
  static constexpr int EPC = 16;
  __device__ static void pack(const float (&v)[EPC], uint4& hi, uint4&) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_fp8x2_storage_t lo2 =
          __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i], v[4 * i + 1]), __NV_SATFINITE, __NV_E4M3);
      const __nv_fp8x2_storage_t hi2 = __nv_cvt_float2_to_fp8x2(
          make_float2(v[4 * i + 2], v[4 * i + 3]), __NV_SATFINITE, __NV_E4M3);
      w[i] = static_cast<uint32_t>(lo2) | (static_cast<uint32_t>(hi2) << 16);
    }
    hi = make_uint4(w[0], w[1], w[2], w[3]);
  }
};

template <>
struct Packer<MODE_TF32> {
  static constexpr int EPC = 4;
  __device__ static void pack(const float (&v)[EPC], uint4& hi, uint4&) {
    hi = make_uint4(tf32_bits(v[0]), tf32_bits(v[1]), tf32_bits(v[2]), tf32_bits(v[3]));
  }
};

template <>
struct Packer<MODE_3XTF32> {
  static constexpr int EPC = 4;
  __device__ static void pack(const float (&v)[EPC], uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = tf32_bits(v[i]);
      l[i] = tf32_bits(v[i] - __uint_as_float(h[i]));  // exact difference, then rounded
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};

}  // namespace pn
