// pp_types.h -- argument blocks of the paper-profile kernels (Tab. 1: odd
// q, one Regev encryption per message bit) and their host-side launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PP_MBITS 256

// q and floor(2^32 / q), for Barrett reduction of 32-bit values
struct ModQ {
  uint32_t q, m;
};

enum { PP_BINOMIAL = 0, PP_GAUSS = 1, PP_UNIFORM = 2 };

struct PpNoiseOut {
  void *out;       // int8 (binomial, Gaussian) or int32 (uniform) samples
  uint32_t count;  // samples
  uint32_t kind;
  uint32_t domain;
  uint32_t pad;
};

struct PpNoiseArgs {
  const uint32_t *rk;  // 44 round-key words (device)
  PpNoiseOut o[3];
  uint32_t nout, clip, kunif, pad;
  uint32_t T[16];      // CDF thresholds (clip used)
};

struct PpAsArgs {
  const uint32_t *A;
  const int8_t *s;   // n
  const int8_t *e;   // n
  uint32_t *t;       // n (pk + 16)
  uint32_t *t2;      // nullable second copy
  uint32_t n;
  ModQ M;
};

struct PpEncArgs {
  const uint32_t *A;
  const int8_t *Rt;    // 256 x n
  const int8_t *E1t;   // 256 x n
  uint32_t *Ut;        // 256 x n (ct)
  uint32_t *flags;
  uint32_t n;
  ModQ M;
};

struct PpVArgs {
  const uint32_t *t;   // n (pk + 16)
  const int8_t *Rt;    // 256 x n
  const int32_t *e2;   // 256
  const uint8_t *m;    // 32 bytes, bit k = bit k % 8 of byte k / 8
  uint32_t *v;         // 256 (ct + 1024 n)
  uint32_t *flags;
  uint32_t n;
  ModQ M;
};

struct PpDecArgs {
  const uint32_t *Ut;  // 256 x n
  const uint32_t *v;   // 256
  const int8_t *s;     // n
  uint32_t *m;         // 8 words = 32 bytes (little-endian bit order)
  uint32_t n;
  ModQ M;
};

void launch_pp_expand_A(const uint8_t *seedA, uint32_t n, ModQ M, uint32_t *A, int num_sms,
                        cudaStream_t st);
void launch_pp_noise(const PpNoiseArgs &a, int num_sms, cudaStream_t st);
void launch_pp_as(const PpAsArgs &a, cudaStream_t st);
void launch_pp_encrypt(const PpEncArgs &a, bool cmp, cudaStream_t st);
void launch_pp_v(const PpVArgs &a, bool cmp, cudaStream_t st);
void launch_pp_decrypt(const PpDecArgs &a, cudaStream_t st);
// A (n x n uint32, entries mod q) -> bf16 limbs [2][n][n] of the GEMM
void launch_pp_limbs(const uint32_t *A, uint32_t n, uint32_t q, uint16_t *limbs, cudaStream_t st);
