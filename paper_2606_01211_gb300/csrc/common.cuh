// common.cuh -- shared device helpers of the LWE KEM library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lwe.h"

#define LWE_DEV __device__ __forceinline__

// Kernel ids used for launch counting and event timing (lwe_kernel_name).
enum LweKernel {
  KID_EXPAND_A = 0,
  KID_NOISE,
  KID_KEYGEN_SEEDS,
  KID_MUL_AS,
  KID_DECRYPT,
  KID_MUL_SA,
  KID_MUL_SA_FUSED,
  KID_V_ENCODE,
  KID_TREE,
  KID_FINAL_KEY,
  KID_DERIVE,
  KID_LIMBS,
  KID_GEMM,
  KID_COUNT
};

// Device-side error word values (set by bounded waits that ran out).
#define LWE_DEVERR_TIMEOUT 1u

LWE_DEV uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

LWE_DEV uint32_t rotl32(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

// 16-byte aligned vector access helpers
LWE_DEV uint4 ld_nc_u4(const void *p) {
  return __ldg(reinterpret_cast<const uint4 *>(p));
}
LWE_DEV uint2 ld_nc_u2(const void *p) {
  return __ldg(reinterpret_cast<const uint2 *>(p));
}

// Packed bytes / halves
LWE_DEV int sext8(uint32_t w, int byte) {
  return (int)(int8_t)(uint8_t)(w >> (8 * byte));
}
