// Conversion of FP32 values into the operand formats of the tensor-core forms.
//
//   TF32    one plane, rounded to nearest (ties away) to 10 mantissa bits
//   BF16    one plane
//   BF16X3  hi = bf16(x), lo = bf16(x - hi): products hi*hi + hi*lo + lo*hi
//   F16X3   hi = fp16(x), lo = fp16(x - hi); operands are kept at |x| <= 1 by
//           power-of-two scaling, so hi never overflows
#pragma once
#include "ofa_internal.cuh"

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Store x at element idx of the hi (and lo) planes of precision prec.
__device__ __forceinline__ void split_store(int prec, void* hi, void* lo, size_t idx, float x) {
  switch (prec) {
    case OFA_PREC_TF32:
      static_cast<float*>(hi)[idx] = tf32_round(x);
      break;
    case OFA_PREC_BF16:
      static_cast<__nv_bfloat16*>(hi)[idx] = __float2bfloat16_rn(x);
      break;
    case OFA_PREC_BF16X3: {
      __nv_bfloat16 h = __float2bfloat16_rn(x);
      static_cast<__nv_bfloat16*>(hi)[idx] = h;
      static_cast<__nv_bfloat16*>(lo)[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
      break;
    }
    case OFA_PREC_F16X3: {
      __half h = __float2half_rn(x);
      static_cast<__half*>(hi)[idx] = h;
      static_cast<__half*>(lo)[idx] = __float2half_rn(x - __half2float(h));
      break;
    }
    default:
      break;
  }
}

// Store the complex pair (re, im) at elements idx, idx+1 (idx even) with one
// 32-bit (16-bit formats) or 64-bit (TF32) store per plane.
__device__ __forceinline__ void split_store2(int prec, void* hi, void* lo, size_t idx, float re,
                                             float im) {
  switch (prec) {
    case OFA_PREC_TF32:
      *reinterpret_cast<float2*>(static_cast<float*>(hi) + idx) =
          make_float2(tf32_round(re), tf32_round(im));
      break;
    case OFA_PREC_BF16:
      *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(hi) + idx) =
          __floats2bfloat162_rn(re, im);
      break;
    case OFA_PREC_BF16X3: {
      __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
      float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(hi) + idx) = h;
      *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(lo) + idx) =
          __floats2bfloat162_rn(re - hf.x, im - hf.y);
      break;
    }
    case OFA_PREC_F16X3: {
      __half2 h = __floats2half2_rn(re, im);
      float2 hf = __half22float2(h);
      *reinterpret_cast<__half2*>(static_cast<__half*>(hi) + idx) = h;
      *reinterpret_cast<__half2*>(static_cast<__half*>(lo) + idx) =
          __floats2half2_rn(re - hf.x, im - hf.y);
      break;
    }
    default:
      break;
  }
}

// Bits of the complex pair (re, im) in the operand format: .x (16-bit formats:
// both halves packed) or .x/.y (TF32); lo is zero for single-plane formats.
__device__ __forceinline__ void split_pack(int prec, float re, float im, uint2& hi, uint2& lo) {
  hi = make_uint2(0u, 0u);
  lo = make_uint2(0u, 0u);
  switch (prec) {
    case OFA_PREC_TF32:
      hi = make_uint2(__float_as_uint(tf32_round(re)), __float_as_uint(tf32_round(im)));
      break;
    case OFA_PREC_BF16: {
      __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
      hi.x = *reinterpret_cast<uint32_t*>(&h);
      break;
    }
    case OFA_PREC_BF16X3: {
      __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
      const float2 hf = __bfloat1622float2(h);
      __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
      hi.x = *reinterpret_cast<uint32_t*>(&h);
      lo.x = *reinterpret_cast<uint32_t*>(&l);
      break;
    }
    case OFA_PREC_F16X3: {
      __half2 h = __floats2half2_rn(re, im);
      const float2 hf = __half22float2(h);
      __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
      hi.x = *reinterpret_cast<uint32_t*>(&h);
      lo.x = *reinterpret_cast<uint32_t*>(&l);
      break;
    }
    default:
      break;
  }
}
