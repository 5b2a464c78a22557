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
  KID_TREE_WARP,
  KID_COUNT
};

// ---- programmatic dependent launch --------------------------------------
// The kernels of the Encaps / Decaps chain are launched with programmatic
// stream serialisation when the context enables it (LWE_OPT_PDL): the next
// kernel of the stream may start while this one drains and run its
// prologue (shared-memory tables, barriers, tensor-memory allocation), then
// waits in pdl_wait() until the previous grid has completed and its memory
// is visible.  Every kernel launched this way calls pdl_wait() in every
// thread before it reads or writes memory that another kernel of the
// stream touches; without the launch attribute both instructions are no-ops.
LWE_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
LWE_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

extern thread_local bool g_launch_pdl;  // set around a context's launches

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = g_launch_pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// The same with thread-block clusters of `cluster` CTAs along x.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k_cluster(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t st, unsigned cluster, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = g_launch_pdl ? 1 : 0;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = cluster;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Device-side error word values (set by bounded waits that ran out).
#define LWE_DEVERR_TIMEOUT 1u

// ---- bounds-checked debug build ------------------------------------------
// Built with -DLWE_CHECK_BOUNDS (build_lib.build(check_bounds=True), the
// library liblwe_check.so), the kernels test the index arithmetic of their
// memory accesses against the sizes they were given: an access that would
// leave its buffer is skipped instead of made, and counted in this
// translation unit's counters with the id of the first failing site
// (lwe_bounds_violations reads and clears them).  A stand-in for a memory
// checker.  In the product build LWE_BOUNDS(cond, site) is `true` and costs
// nothing.
#ifdef LWE_CHECK_BOUNDS
static __device__ unsigned long long g_bounds_bad;
static __device__ unsigned int g_bounds_site;
LWE_DEV bool lwe_in_bounds(bool ok, unsigned site) {
  if (!ok && atomicAdd(&g_bounds_bad, 1ull) == 0ull) g_bounds_site = site;
  return ok;
}
#define LWE_BOUNDS(cond, site) lwe_in_bounds((cond), (site))
// host: read and clear this translation unit's counters
#define LWE_BOUNDS_READER(fn)                                                          \
  cudaError_t fn(unsigned long long *count, unsigned *site) {                          \
    unsigned long long zero = 0;                                                       \
    cudaError_t e = cudaMemcpyFromSymbol(count, g_bounds_bad, sizeof *count);          \
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(site, g_bounds_site, sizeof *site); \
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds_bad, &zero, sizeof zero);    \
    return e;                                                                          \
  }
#else
#define LWE_BOUNDS(cond, site) true
#define LWE_BOUNDS_READER(fn)                                     \
  cudaError_t fn(unsigned long long *count, unsigned *site) {     \
    *count = 0;                                                   \
    *site = 0;                                                    \
    return cudaSuccess;                                           \
  }
#endif

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
