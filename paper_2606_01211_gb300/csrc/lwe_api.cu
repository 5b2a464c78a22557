// lwe_api.cu -- host runtime behind the C ABI of include/lwe.h.
//
// Owns the parameter presets, the noise table, the AES table upload, the
// contexts and their device workspaces, and the order of kernel launches
// that makes up KeyGen, Encaps and Decaps (Alg. 1, 4, 5 of the paper).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lwe.h"
#include "common.cuh"
#include "gemm_tc.h"
#include "kem_kernels.h"
#include "pp_types.h"
#include "../../include/lwe_pp.h"

namespace {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return LWE_ECUDA;
}

#define CUDA_TRY(x)                                 \
  do {                                              \
    cudaError_t _e = (x);                           \
    if (_e != cudaSuccess) return cuda_fail(_e);    \
  } while (0)

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// An NVTX range around each work-enqueuing entry point, named after it, so
// that a timeline profiler shows which library call issued which kernels
// (no cost beyond a function-pointer call when no profiler is attached).
struct NvtxScope {
  explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
};
#define LWE_TRACE(name) NvtxScope _nvtx_scope(name)

// ---- AES round table T0, from the S-box of FIPS-197 ---------------------
// S(x) = affine(x^-1) with the inverse taken through log / antilog tables
// of the generator 3 of GF(2^8)*; T0[x] = 2S | S<<8 | S<<16 | 3S<<24.
uint8_t gmul2(uint8_t a) { return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0)); }

void build_aes_T0(uint32_t T0[256]) {
  uint8_t alog[256], logt[256];
  uint8_t x = 1;
  for (int i = 0; i < 255; i++) {
    alog[i] = x;
    logt[x] = (uint8_t)i;
    x = (uint8_t)(x ^ gmul2(x));  // multiply by 3
  }
  for (int v = 0; v < 256; v++) {
    uint8_t inv = v == 0 ? 0 : alog[(255 - logt[v]) % 255];
    uint8_t s = inv;
    for (int r = 1; r <= 4; r++) s ^= (uint8_t)((inv << r) | (inv >> (8 - r)));
    s ^= 0x63;
    uint8_t s2 = gmul2(s), s3 = (uint8_t)(s2 ^ s);
    T0[v] = (uint32_t)s2 | ((uint32_t)s << 8) | ((uint32_t)s << 16) | ((uint32_t)s3 << 24);
  }
}

// ---- per-device one-time set-up ------------------------------------------
std::mutex g_dev_mu;
bool g_dev_ready[128];

int device_setup(int device) {
  if (device < 0 || device >= 128) return LWE_EINVAL;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_dev_ready[device]) return LWE_OK;
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) return LWE_EUNSUPPORTED;
  int prev = 0;
  CUDA_TRY(cudaGetDevice(&prev));
  CUDA_TRY(cudaSetDevice(device));
  uint32_t T0[256];
  build_aes_T0(T0);
  cudaError_t e = lwe_upload_aes_table(T0);
  if (e == cudaSuccess) e = lwe_kernel_smem_setup();
  if (e == cudaSuccess) e = lwe_gemm_setup();
  cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e);
  g_dev_ready[device] = true;
  return LWE_OK;
}

int current_device_setup(int *dev_out, int *sms_out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  int rc = device_setup(dev);
  if (rc != LWE_OK) return rc;
  if (dev_out) *dev_out = dev;
  if (sms_out) CUDA_TRY(cudaDeviceGetAttribute(sms_out, cudaDevAttrMultiProcessorCount, dev));
  return LWE_OK;
}

// ---- noise table (independent restatement of the rounded Gaussian) -------
double norm_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

int cdf_table(double sigma, uint32_t clip, uint16_t T[16]) {
  if (!(sigma > 0.0) || clip < 1 || clip > 15) return LWE_EINVAL;
  double mass[16];
  double z = 0.0;
  for (uint32_t k = 0; k <= clip; k++) {
    mass[k] = norm_cdf((k + 0.5) / sigma) - norm_cdf((k - 0.5) / sigma);
    z += k ? 2.0 * mass[k] : mass[k];
  }
  double acc = 0.0;
  for (uint32_t k = 0; k < 16; k++) T[k] = 0x7fff;
  for (uint32_t k = 0; k < clip; k++) {
    acc += (k ? 2.0 * mass[k] : mass[k]) / z;
    const double v = std::floor(acc * 32768.0 + 0.5) - 1.0;
    if (v < 0.0 || v >= 32767.0) return LWE_EINVAL;
    T[k] = (uint16_t)v;
    if (k > 0 && T[k] <= T[k - 1]) return LWE_EINVAL;
  }
  return LWE_OK;
}

int params_check(const lwe_params *p) {
  if (!p) return LWE_EINVAL;
  if (p->n < 16 || p->n > 65536 || (p->n % 16) != 0) return LWE_EINVAL;
  if (p->nbar != 8 || p->mbar != 8) return LWE_EINVAL;
  if (p->logq < 2 || p->logq > 16) return LWE_EINVAL;
  if (p->B < 1 || p->B > 4 || p->B >= p->logq) return LWE_EINVAL;
  uint16_t T[16];
  return cdf_table(p->sigma, p->clip, T);
}

size_t pk_bytes(const lwe_params &p) { return 16 + 16 * (size_t)p.n; }
size_t sk_bytes(const lwe_params &p) { return 8 * (size_t)p.n + 64 + pk_bytes(p); }
size_t ct_bytes(const lwe_params &p) { return 16 * (size_t)p.n + 128; }
uint32_t mu_bytes(const lwe_params &p) { return 8 * p.B; }

const char *kKernelNames[KID_COUNT] = {
    "k_expand_A", "k_noise",    "k_keygen_seeds", "k_mul_as", "k_decrypt",
    "k_sa",       "k_sa_fused", "k_v_encode",     "k_tree",   "k_final_key",
    "k_derive",   "k_limbs",    "k_gemm_tc",      "k_tree_warp"};

}  // namespace

thread_local bool g_launch_pdl = false;

// ---- context ---------------------------------------------------------------
struct TimedLaunch {
  int kid;
  cudaEvent_t a, b;
};

struct lwe_ctx {
  lwe_params p;
  uint16_t T[16];
  int device = 0;
  int num_sms = 0;
  uint32_t max_batch = 0;
  int path = LWE_PATH_AUTO;
  int tensor_min = 64;
  int gemm_bn = 128;
  int gemm_pair = 1;
  uint32_t gemm_group = 0;  // LWE_OPT_GEMM_GROUP; 0: chosen per launch
  int8_t *ntab = nullptr;    // the sampler table for T (64 KB), built at creation
  uint64_t *tdig = nullptr;  // leaf digests of long tree hashes (n >= 4096)
  uint64_t tdig_words = 0;
  bool serial = false;  // LWE_OPT_SERIAL: side-stream work on the caller's stream
  bool pdl = true;      // LWE_OPT_PDL
  int64_t tree_warp_max = -1;  // LWE_OPT_WARP_HASH_MAX; -1: the number of SMs
  bool timing = false;
  uint64_t launches = 0;
  std::vector<TimedLaunch> pending;
  std::vector<TimedLaunch> replay;  // pairs captured into a CUDA graph
  std::vector<cudaEvent_t> free_events;
  uint64_t stat_launches[KID_COUNT] = {};
  double stat_ms[KID_COUNT] = {};
  // workspace
  uint8_t *ws = nullptr;
  size_t ws_bytes = 0;
  uint8_t *seeds = nullptr, *mu = nullptr, *kp = nullptr, *pkh = nullptr;
  uint8_t *hc = nullptr;       // H(c) per item (Decaps)
  uint32_t *flags = nullptr, *dev_err = nullptr;
  uint32_t *rk = nullptr;     // 44 AES round-key words per item
  uint8_t *pkhs = nullptr;    // H(pk) per item (multi-key Encaps)
  int8_t *sp8 = nullptr, *ep8 = nullptr, *epp = nullptr;
  uint16_t *spbf = nullptr;  // bf16 bits
  uint16_t *limbs = nullptr; // bf16 bits, [2][n + 8][n]
  uint16_t *partial = nullptr; // K-split running sums, [8 max_batch][n + 8]
  uint32_t kchunk = 0;         // exact K per GEMM pass
  bool has_tensor = false;
  // the key bound by lwe_ctx_bind_key: its buffers, H(pk) (bpkh) and
  // whether `limbs` still holds the limb split of its [A | B]
  bool bound = false;
  const uint8_t *bound_pk = nullptr, *bound_sk = nullptr;
  const uint16_t *bound_A = nullptr;
  uint8_t *bpkh = nullptr;
  bool limbs_bound = false;
  // side stream for work independent of the re-encryption (Decaps' H(c))
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_limbs = nullptr;
};

namespace {

cudaEvent_t take_event(lwe_ctx *c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// hashing launches of at most this many items use one Keccak state per warp
uint32_t warp_hash_max(const lwe_ctx *c) {
  return c->tree_warp_max < 0 ? (uint32_t)c->num_sms : (uint32_t)c->tree_warp_max;
}

struct LaunchScope {
  lwe_ctx *c;
  int kid;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  unsigned flags = cudaEventRecordDefault;
  bool pdl_before = g_launch_pdl;
  LaunchScope(lwe_ctx *c_, int kid_, cudaStream_t st_) : c(c_), kid(kid_), st(st_) {
    // per-launch event timing brackets each kernel, so it launches plainly
    g_launch_pdl = c && c->pdl && !c->timing;
    if (c && c->timing) {
      a = take_event(c);
      b = take_event(c);
      // inside a stream capture the records must become event-record nodes
      // of the graph (re-recorded by every replay), not capture dependencies
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        flags = cudaEventRecordExternal;
      if (a && b) cudaEventRecordWithFlags(a, st, flags);
    }
  }
  ~LaunchScope() {
    g_launch_pdl = pdl_before;
    if (!c) return;
    c->launches++;
    if (a && b) {
      cudaEventRecordWithFlags(b, st, flags);
      c->pending.push_back({kid, a, b});
    }
  }
};

#define LAUNCH(ctx, kid, stream, call) \
  do {                                 \
    LaunchScope _ls(ctx, kid, stream); \
    call;                              \
  } while (0)

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  return LWE_OK;
}

void harvest(lwe_ctx *c) {
  for (auto &t : c->pending) {
    cudaEventSynchronize(t.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      c->stat_launches[t.kid]++;
      c->stat_ms[t.kid] += ms;
    }
    c->free_events.push_back(t.a);
    c->free_events.push_back(t.b);
  }
  c->pending.clear();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

NoiseArgs noise_args(const lwe_ctx *c, uint32_t count) {
  NoiseArgs a;
  memset(&a, 0, sizeof a);
  a.rk = c->rk;
  a.count = count;
  for (int i = 0; i < 16; i++) a.T[i] = c->T[i];
  a.tab_img = reinterpret_cast<const uint4 *>(c->ntab);
  return a;
}

NoiseOut noise_out(void *base, uint64_t item_stride, uint32_t nsamples, uint32_t domain,
                   uint32_t fmt) {
  const uint32_t nblk = (nsamples + 7) / 8;
  return NoiseOut{base, item_stride, nsamples, domain, fmt, (nblk + NOISE_RUN - 1) / NOISE_RUN};
}

void noise_finish(NoiseArgs &a) {
  a.runs_per_item = 0;
  for (uint32_t s = 0; s < a.nout; s++) a.runs_per_item += a.out[s].runs;
}

DeriveArgs derive_args(const lwe_ctx *c, const uint8_t *coins, const uint8_t *pkh,
                       uint32_t count) {
  DeriveArgs d;
  memset(&d, 0, sizeof d);
  d.coins = coins;
  d.pkh = pkh;
  d.mu = c->mu;
  d.kprime = c->kp;
  d.seeds = c->seeds;
  d.rk = c->rk;
  d.count = count;
  d.mu_bytes = mu_bytes(c->p);
  return d;
}

DecryptArgs decrypt_args(const lwe_ctx *c, const uint8_t *ct, const int8_t *St,
                         const uint8_t *const *sk_ptrs) {
  DecryptArgs d;
  memset(&d, 0, sizeof d);
  d.ct = ct;
  d.ct_bytes = ct_bytes(c->p);
  d.St = St;
  d.sk_ptrs = sk_ptrs;
  d.mu = c->mu;
  d.n = c->p.n;
  d.logq = c->p.logq;
  d.B = c->p.B;
  return d;
}

// Encrypt (Alg. 2) for `count` items whose seedSE' and mu are in the
// workspace; writes ct, or (cmp) compares against ct and sets flags.
// Per-item key material of the multi-key calls: item e's key object is
// ptrs[e] (its public key at ptrs[e] + pk_off), its stored A is A_ptrs[e]
// (A_ptrs NULL: every item regenerates A from its seed).
struct ItemKeys {
  const uint8_t *const *ptrs = nullptr;
  uint64_t pk_off = 0;
  const uint16_t *const *A_ptrs = nullptr;
};

// The stream for work that does not depend on the main chain (the tensor
// path's limbs, Decaps' H(c)): the context's side stream, or the caller's
// stream when LWE_OPT_SERIAL is set.
cudaStream_t side_stream(const lwe_ctx *c, cudaStream_t st) { return c->serial ? st : c->side; }

// Whether a call of `count` items runs its product on the tensor cores.
bool use_tensor(const lwe_ctx *c, uint32_t count, const ItemKeys *ik) {
  bool tensor = false;
  if (c->path == LWE_PATH_TENSOR)
    tensor = true;
  else if (c->path == LWE_PATH_AUTO)
    tensor = (int)count >= c->tensor_min;
  return tensor && c->has_tensor && !ik;  // one GEMM needs one shared A
}

// The GEMM's B operand: limbs of the columns of [A | B] (A stored, or
// regenerated from seedA = pk[0:16]).  Depends on the key only.
void launch_limbs(lwe_ctx *c, const uint8_t *pk, const uint16_t *A, cudaStream_t st,
                  bool for_bound = false) {
  c->limbs_bound = for_bound;
  GemmLimbArgs la;
  la.A = A;
  la.seedA = pk;
  la.B = pk + 16;
  la.n = c->p.n;
  la.logq = c->p.logq;
  la.limbs = c->limbs;
  LAUNCH(c, KID_LIMBS, st, launch_gemm_limbs(la, c->num_sms, st));
}

// Where the tensor path's limbs come from: made here on the main stream,
// made by the caller on the side stream (ev_limbs), or already in place (the
// bound key's).
enum LimbsFrom { LIMBS_HERE = 0, LIMBS_SIDE = 1, LIMBS_READY = 2 };

int run_encrypt(lwe_ctx *c, const uint8_t *pk, const uint16_t *A, uint32_t count, uint8_t *ct,
                bool cmp, cudaStream_t st, const ItemKeys *ik = nullptr,
                int limbs_from = LIMBS_HERE) {
  const uint32_t n = c->p.n;
  const bool tensor = use_tensor(c, count, ik);

  NoiseArgs na = noise_args(c, count);
  na.nout = 3;
  if (tensor)
    na.out[0] = noise_out(c->spbf, 16ull * n, 8 * n, 3, NOISE_BF16);
  else
    na.out[0] = noise_out(c->sp8, 8ull * n, 8 * n, 3, NOISE_I8);
  na.out[1] = noise_out(c->ep8, 8ull * n, 8 * n, 4, NOISE_I8);
  na.out[2] = noise_out(c->epp, 64, 64, 5, NOISE_I8);
  noise_finish(na);
  LAUNCH(c, KID_NOISE, st, launch_noise(na, c->num_sms, st));

  if (tensor) {
    if (limbs_from == LIMBS_SIDE)  // made on the side stream by the caller
      CUDA_TRY(cudaStreamWaitEvent(st, c->ev_limbs, 0));
    else if (limbs_from == LIMBS_HERE)
      launch_limbs(c, pk, A, st);
    GemmSaArgs ga;
    memset(&ga, 0, sizeof ga);
    ga.S = c->spbf;
    ga.limbs = c->limbs;
    ga.E = c->ep8;
    ga.Epp = c->epp;
    ga.mu = c->mu;
    ga.out = ct;
    ga.out_stride = ct_bytes(c->p);
    ga.flags = c->flags;
    ga.dev_err = c->dev_err;
    ga.n = n;
    ga.ncols = n + 8;
    ga.rows = 8 * count;
    ga.logq = c->p.logq;
    ga.B = c->p.B;
    ga.cmp = cmp ? 1 : 0;
    ga.bn = c->gemm_bn;
    ga.pair = c->gemm_pair;
    ga.group_m = c->gemm_group;
    ga.clip = c->p.clip;
    ga.kchunk = c->kchunk;
    ga.partial_out = c->partial;
    int rc = LWE_OK;
    LAUNCH(c, KID_GEMM, st, rc = launch_gemm_sa(ga, c->num_sms, st));
    if (rc != LWE_OK) return rc;
    return check_launch();
  }

  MulSaArgs sa;
  memset(&sa, 0, sizeof sa);
  sa.A = A;
  sa.seedA = pk;
  sa.n = n;
  sa.logq = c->p.logq;
  sa.S = c->sp8;
  sa.s_stride = 8ull * n;
  sa.E = c->ep8;
  sa.e_stride = 8ull * n;
  sa.out = ct;
  sa.out_stride = ct_bytes(c->p);
  sa.flags = c->flags;
  bool fused = A == nullptr;
  if (ik) {
    sa.A_ptrs = ik->A_ptrs;
    sa.seed_ptrs = ik->ptrs;
    sa.seed_off = ik->pk_off;
    fused = ik->A_ptrs == nullptr;
  }
  LAUNCH(c, fused ? KID_MUL_SA_FUSED : KID_MUL_SA, st, launch_mul_sa(sa, count, fused, cmp, c->num_sms, st));

  VEncArgs va;
  memset(&va, 0, sizeof va);
  va.pk = pk;
  if (ik) {
    va.pk_ptrs = ik->ptrs;
    va.pk_off = ik->pk_off;
  }
  va.S = c->sp8;
  va.s_stride = 8ull * n;
  va.Epp = c->epp;
  va.epp_stride = 64;
  va.mu = c->mu;
  va.ct = ct;
  va.ct_bytes = ct_bytes(c->p);
  va.flags = c->flags;
  va.n = n;
  va.logq = c->p.logq;
  va.B = c->p.B;
  LAUNCH(c, KID_V_ENCODE, st, launch_v_encode(va, count, cmp, st));
  return check_launch();
}

void tree_hash(lwe_ctx *c, const uint8_t *msgs, uint64_t stride, uint32_t len, uint32_t count,
               int mode, uint8_t *out, uint64_t out_stride, uint8_t *out2, uint64_t out2_stride,
               cudaStream_t st, const uint8_t *const *msg_ptrs = nullptr) {
  TreeArgs ta;
  memset(&ta, 0, sizeof ta);
  ta.msgs = msgs;
  ta.msg_ptrs = msg_ptrs;
  ta.stride = stride;
  ta.len = len;
  ta.count = count;
  ta.mode = mode;
  ta.out = out;
  ta.out_stride = out_stride;
  ta.out2 = out2;
  ta.out2_stride = out2_stride;
  ta.kprime = c->kp;
  ta.dig = c->tdig;
  ta.dig_words = c->tdig_words;
  const uint32_t warp_max = warp_hash_max(c);
  LAUNCH(c, count <= warp_max ? KID_TREE_WARP : KID_TREE, st,
         launch_tree(ta, c->num_sms, warp_max, st));
}

int hash_tree(lwe_ctx *c, const uint8_t *msgs, uint64_t stride, uint32_t len, uint32_t count,
              int mode, uint8_t *out, uint64_t out_stride, uint8_t *out2, uint64_t out2_stride,
              cudaStream_t st) {
  tree_hash(c, msgs, stride, len, count, mode, out, out_stride, out2, out2_stride, st);
  return check_launch();
}

// Decaps' final key from K', H(c) and the re-encryption flags
void final_key(lwe_ctx *c, const uint8_t *z, const uint8_t *const *z_ptrs, uint64_t z_off,
               uint32_t count, uint8_t *K, cudaStream_t st) {
  FinalKeyArgs fa;
  memset(&fa, 0, sizeof fa);
  fa.kprime = c->kp;
  fa.hc = c->hc;
  fa.z = z;
  fa.z_ptrs = z_ptrs;
  fa.z_off = z_off;
  fa.flags = c->flags;
  fa.K = K;
  fa.count = count;
  LAUNCH(c, KID_FINAL_KEY, st, launch_final_key(fa, warp_hash_max(c), st));
}

int set_device_of(lwe_ctx *c) {
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != c->device) CUDA_TRY(cudaSetDevice(c->device));
  return LWE_OK;
}

}  // namespace

// ---- built-in scratch of lwe_encaps_noalloc ------------------------------
// One fixed area per device, compiled into the library.  Host code must not
// pass `g_noalloc_scratch` itself to a kernel (on the host it names a
// stand-in, not device memory): its device address is looked up once per
// device with cudaGetSymbolAddress while that device is current.
static __device__ __align__(256) uint8_t g_noalloc_scratch[LWE_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
uint8_t *g_noalloc_addr[128];

int noalloc_scratch(int dev, uint8_t **out) {
  if (dev < 0 || dev >= 128) return LWE_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    g_noalloc_addr[dev] = static_cast<uint8_t *>(ptr);
  }
  *out = g_noalloc_addr[dev];
  return LWE_OK;
}

}  // namespace

extern "C" {

int lwe_params_preset(int id, lwe_params *out) {
  if (!out) return LWE_EINVAL;
  static const struct {
    uint32_t n, logq, B, clip;
    double sigma;
  } P[] = {{640, 15, 2, 12, 2.8},  {976, 16, 3, 10, 2.3},   {1344, 16, 4, 6, 1.4},
           {4096, 16, 2, 12, 2.8}, {16384, 16, 1, 12, 2.8}, {32768, 16, 1, 12, 2.8}};
  if (id < 0 || id >= (int)(sizeof P / sizeof P[0])) return LWE_EINVAL;
  out->n = P[id].n;
  out->nbar = 8;
  out->mbar = 8;
  out->logq = P[id].logq;
  out->B = P[id].B;
  out->clip = P[id].clip;
  out->sigma = P[id].sigma;
  return LWE_OK;
}

int lwe_params_check(const lwe_params *p) { return params_check(p); }

int lwe_cdf_table(const lwe_params *p, uint16_t T[16]) {
  if (!p || !T) return LWE_EINVAL;
  return cdf_table(p->sigma, p->clip, T);
}

size_t lwe_pk_bytes(const lwe_params *p) { return p ? pk_bytes(*p) : 0; }
size_t lwe_sk_bytes(const lwe_params *p) { return p ? sk_bytes(*p) : 0; }
size_t lwe_ct_bytes(const lwe_params *p) { return p ? ct_bytes(*p) : 0; }

int lwe_ctx_create(const lwe_params *p, uint32_t max_batch, int device, lwe_ctx **out) {
  if (!out) return LWE_EINVAL;
  *out = nullptr;
  if (params_check(p) != LWE_OK || max_batch < 1) return LWE_EINVAL;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return LWE_EINVAL;
  int rc = device_setup(device);
  if (rc != LWE_OK) return rc;
  int prev = 0;
  CUDA_TRY(cudaGetDevice(&prev));
  CUDA_TRY(cudaSetDevice(device));

  lwe_ctx *c = new lwe_ctx();
  c->p = *p;
  cdf_table(p->sigma, p->clip, c->T);
  c->device = device;
  c->max_batch = max_batch;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);

  const size_t n = p->n;
  const size_t Bm = max_batch;
  // tensor path workspaces (bf16 S', limbs, K-split sums) are sized for
  // batched use: always for n <= 8192, and for larger n when max_batch >= 64
  c->has_tensor = lwe_gemm_supported(p->n, p->logq, p->clip) && (p->n <= 8192 || max_batch >= 64);
  c->kchunk = lwe_gemm_kchunk(p->clip);
  const bool ksplit = c->has_tensor;  // the K-split buffer also serves LWE_OPT_GEMM_KCHUNK
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_seeds = carve(32 * Bm), o_mu = carve(32 * Bm), o_kp = carve(32 * Bm);
  const size_t o_flags = carve(4 * Bm), o_err = carve(16), o_pkh = carve(32);
  const size_t o_bpkh = carve(32);
  const size_t o_rk = carve(176 * Bm), o_pkhs = carve(32 * Bm);
  const size_t o_hc = carve(32 * Bm), o_ntab = carve(65536);
  const size_t o_sp8 = carve(8 * n * Bm), o_ep8 = carve(8 * n * Bm), o_epp = carve(64 * Bm);
  // tree hashes of messages of more than 32 chunks keep their leaf digests
  // in global memory (32 bytes per chunk)
  const size_t tchunks = (std::max(ct_bytes(*p), pk_bytes(*p)) + LWE_TREE_CHUNK - 1) / LWE_TREE_CHUNK;
  const size_t tdig_bytes = tchunks > 32 ? 32 * tchunks * Bm : 0;
  const size_t o_tdig = tdig_bytes ? carve(tdig_bytes) : 0;
  size_t o_spbf = 0, o_limbs = 0;
  size_t o_partial = 0;
  if (c->has_tensor) {
    o_spbf = carve(16 * n * Bm);
    o_limbs = carve(2 * 2 * (n + 8) * n);
    if (ksplit) o_partial = carve(2 * 8 * Bm * (n + 8));
  }
  c->ws_bytes = off;
  cudaError_t e = cudaMalloc(&c->ws, c->ws_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    cudaSetDevice(prev);
    return LWE_ENOMEM;
  }
  c->seeds = c->ws + o_seeds;
  c->mu = c->ws + o_mu;
  c->kp = c->ws + o_kp;
  c->flags = reinterpret_cast<uint32_t *>(c->ws + o_flags);
  c->dev_err = reinterpret_cast<uint32_t *>(c->ws + o_err);
  c->rk = reinterpret_cast<uint32_t *>(c->ws + o_rk);
  c->pkhs = c->ws + o_pkhs;
  c->pkh = c->ws + o_pkh;
  c->bpkh = c->ws + o_bpkh;
  c->hc = c->ws + o_hc;
  c->ntab = reinterpret_cast<int8_t *>(c->ws + o_ntab);
  c->sp8 = reinterpret_cast<int8_t *>(c->ws + o_sp8);
  c->ep8 = reinterpret_cast<int8_t *>(c->ws + o_ep8);
  c->epp = reinterpret_cast<int8_t *>(c->ws + o_epp);
  if (tdig_bytes) {
    c->tdig = reinterpret_cast<uint64_t *>(c->ws + o_tdig);
    c->tdig_words = tdig_bytes / 8;
  }
  if (c->has_tensor) {
    c->spbf = reinterpret_cast<uint16_t *>(c->ws + o_spbf);
    c->limbs = reinterpret_cast<uint16_t *>(c->ws + o_limbs);
    if (ksplit) c->partial = reinterpret_cast<uint16_t *>(c->ws + o_partial);
  }
  e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_limbs, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(c->ws, 0, c->ws_bytes);
  if (e == cudaSuccess) {
    NoiseArgs na = noise_args(c, 0);
    na.tab_img = nullptr;
    launch_noise_table(na, c->ntab, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_limbs) cudaEventDestroy(c->ev_limbs);
    if (c->side) cudaStreamDestroy(c->side);
    cudaFree(c->ws);
    delete c;
    return cuda_fail(e);
  }
  *out = c;
  return LWE_OK;
}

int lwe_ctx_destroy(lwe_ctx *c) {
  if (!c) return LWE_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (auto &t : c->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto &t : c->replay) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : c->free_events) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_limbs) cudaEventDestroy(c->ev_limbs);
  if (c->side) cudaStreamDestroy(c->side);
  cudaFree(c->ws);
  cudaSetDevice(prev);
  delete c;
  return LWE_OK;
}

int lwe_ctx_set_option(lwe_ctx *c, int option, int64_t value) {
  if (!c) return LWE_EINVAL;
  switch (option) {
    case LWE_OPT_PATH:
      if (value < LWE_PATH_AUTO || value > LWE_PATH_TENSOR) return LWE_EINVAL;
      if (value == LWE_PATH_TENSOR && !c->has_tensor) return LWE_EUNSUPPORTED;
      c->path = (int)value;
      return LWE_OK;
    case LWE_OPT_TENSOR_MIN:
      if (value < 1) return LWE_EINVAL;
      c->tensor_min = (int)value;
      return LWE_OK;
    case LWE_OPT_TIMING:
      c->timing = value != 0;
      return LWE_OK;
    case LWE_OPT_GEMM_BN:
      if (value != 64 && value != 128) return LWE_EINVAL;
      c->gemm_bn = (int)value;
      return LWE_OK;
    case LWE_OPT_SERIAL:
      c->serial = value != 0;
      return LWE_OK;
    case LWE_OPT_GEMM_PAIR:
      if (value != 0 && value != 1) return LWE_EINVAL;
      c->gemm_pair = (int)value;
      return LWE_OK;
    case LWE_OPT_PDL:
      if (value != 0 && value != 1) return LWE_EINVAL;
      c->pdl = value != 0;
      return LWE_OK;
    case LWE_OPT_GEMM_GROUP:
      if (value < 0 || value > 64) return LWE_EINVAL;
      c->gemm_group = (uint32_t)value;
      return LWE_OK;
    case LWE_OPT_WARP_HASH_MAX:
      if (value < -1 || value > 0xffffffffLL) return LWE_EINVAL;
      c->tree_warp_max = value;
      return LWE_OK;
    case LWE_OPT_GEMM_KCHUNK:
      if (value == 0) {
        c->kchunk = lwe_gemm_kchunk(c->p.clip);
        return LWE_OK;
      }
      if (value < 64 || (value % 64) || value > (int64_t)lwe_gemm_kchunk(c->p.clip))
        return LWE_EINVAL;
      c->kchunk = (uint32_t)value;
      return LWE_OK;
    default:
      return LWE_EINVAL;
  }
}

int lwe_keygen(lwe_ctx *c, const uint8_t *seeds, uint32_t count, uint8_t *pk, uint8_t *sk,
               uint16_t *A_out, void *stream) {
  LWE_TRACE("lwe_keygen");
  if (!c) return LWE_EINVAL;
  if (count == 0) return LWE_OK;
  if (count > c->max_batch) return LWE_ECAPACITY;
  if (!seeds || !pk || !sk || !aligned16(seeds) || !aligned16(pk) || !aligned16(sk) ||
      (A_out && !aligned16(A_out)))
    return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_params &p = c->p;
  const uint32_t n = p.n;
  const size_t pkb = pk_bytes(p), skb = sk_bytes(p);

  KeygenSeedArgs ka{seeds, pk, sk, c->seeds, c->rk, pkb, skb, 8ull * n, 8ull * n + 64, count, 0};
  LAUNCH(c, KID_KEYGEN_SEEDS, st, launch_keygen_seeds(ka, warp_hash_max(c), st));

  NoiseArgs na = noise_args(c, count);
  na.nout = 2;
  na.out[0] = noise_out(sk, skb, 8 * n, 1, NOISE_I8);           // S^T, row-major 8 x n
  na.out[1] = noise_out(c->ep8, 8ull * n, 8 * n, 2, NOISE_I8);  // E, n x 8
  noise_finish(na);
  LAUNCH(c, KID_NOISE, st, launch_noise(na, c->num_sms, st));

  if (A_out)
    LAUNCH(c, KID_EXPAND_A, st,
           launch_expand_A(c->seeds, 32, count, n, p.logq, A_out, (uint64_t)n * n, c->num_sms, st));

  MulAsArgs ma;
  memset(&ma, 0, sizeof ma);
  ma.A = A_out;
  ma.a_stride = (uint64_t)n * n;
  ma.seeds = c->seeds;
  ma.seed_stride = 32;
  ma.n = n;
  ma.logq = p.logq;
  ma.St = reinterpret_cast<const int8_t *>(sk);
  ma.st_stride = skb;
  ma.E = c->ep8;
  ma.e_stride = 8ull * n;
  ma.out = pk + 16;
  ma.out_stride = pkb;
  ma.out2 = sk + 8 * (size_t)n + 64 + 16;
  ma.out2_stride = skb;
  LAUNCH(c, KID_MUL_AS, st, launch_mul_as(ma, count, A_out == nullptr, c->num_sms, st));

  // H(pk) into sk
  return hash_tree(c, pk, pkb, (uint32_t)pkb, count, TREE_DIGEST, sk + 8 * (size_t)n + 32, skb,
                   nullptr, 0, st);
}

int lwe_encaps(lwe_ctx *c, const uint8_t *pk, const uint16_t *A, const uint8_t *coins,
               uint32_t count, uint8_t *ct, uint8_t *K, void *stream) {
  LWE_TRACE("lwe_encaps");
  if (!c) return LWE_EINVAL;
  if (count == 0) return LWE_OK;
  if (count > c->max_batch) return LWE_ECAPACITY;
  if (!pk || !coins || !ct || !K || !aligned16(pk) || !aligned16(coins) || !aligned16(ct) ||
      !aligned16(K) || (A && !aligned16(A)))
    return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_params &p = c->p;
  const size_t pkb = pk_bytes(p), ctb = ct_bytes(p);

  // The bound key's H(pk) and limbs are made once, at lwe_ctx_bind_key.
  // Otherwise, on the tensor path, the limbs of [A | B] are made on the side
  // stream while the main stream hashes pk (one message: a latency-bound
  // launch).
  const bool bound = c->bound && pk == c->bound_pk && A == c->bound_A;
  const bool tensor = use_tensor(c, count, nullptr);
  int limbs_from = LIMBS_HERE;
  if (tensor && bound && c->limbs_bound) {
    limbs_from = LIMBS_READY;
  } else if (tensor) {
    cudaStream_t ss = side_stream(c, st);
    CUDA_TRY(cudaEventRecord(c->ev_fork, st));
    CUDA_TRY(cudaStreamWaitEvent(ss, c->ev_fork, 0));
    launch_limbs(c, pk, A, ss, bound);
    CUDA_TRY(cudaEventRecord(c->ev_limbs, ss));
    limbs_from = LIMBS_SIDE;
  }
  const uint8_t *pkh = c->bpkh;
  if (!bound) {
    rc = hash_tree(c, pk, pkb, (uint32_t)pkb, 1, TREE_DIGEST, c->pkh, 32, nullptr, 0, st);
    if (rc) return rc;
    pkh = c->pkh;
  }
  DeriveArgs da = derive_args(c, coins, pkh, count);
  LAUNCH(c, KID_DERIVE, st, launch_derive(da, warp_hash_max(c), st));
  rc = run_encrypt(c, pk, A, count, ct, false, st, nullptr, limbs_from);
  if (rc) return rc;
  return hash_tree(c, ct, ctb, (uint32_t)ctb, count, TREE_ENC_KEY, K, 32, nullptr, 0, st);
}

int lwe_decaps(lwe_ctx *c, const uint8_t *sk, const uint16_t *A, const uint8_t *ct,
               uint32_t count, uint8_t *K, void *stream) {
  LWE_TRACE("lwe_decaps");
  if (!c) return LWE_EINVAL;
  if (count == 0) return LWE_OK;
  if (count > c->max_batch) return LWE_ECAPACITY;
  if (!sk || !ct || !K || !aligned16(sk) || !aligned16(ct) || !aligned16(K) ||
      (A && !aligned16(A)))
    return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_params &p = c->p;
  const uint32_t n = p.n;
  const size_t ctb = ct_bytes(p);
  const uint8_t *z = sk + 8 * (size_t)n;
  const uint8_t *pkh = z + 32;
  const uint8_t *pk = pkh + 32;

  CUDA_TRY(cudaMemsetAsync(c->flags, 0, 4 * (size_t)count, st));
  // H(c) does not depend on the re-encryption: it runs on the side stream,
  // overlapping the re-encryption, and joins before the key selection (the
  // tensor path's limbs go first on that stream)
  cudaStream_t ss = side_stream(c, st);
  CUDA_TRY(cudaEventRecord(c->ev_fork, st));
  CUDA_TRY(cudaStreamWaitEvent(ss, c->ev_fork, 0));
  const bool bound = c->bound && sk == c->bound_sk && A == c->bound_A;
  const bool tensor = use_tensor(c, count, nullptr);
  int limbs_from = LIMBS_HERE;
  if (tensor && bound && c->limbs_bound) {
    limbs_from = LIMBS_READY;
  } else if (tensor) {
    launch_limbs(c, pk, A, ss, bound);
    CUDA_TRY(cudaEventRecord(c->ev_limbs, ss));
    limbs_from = LIMBS_SIDE;
  }
  tree_hash(c, ct, ctb, (uint32_t)ctb, count, TREE_DIGEST, c->hc, 32, nullptr, 0, ss);
  CUDA_TRY(cudaEventRecord(c->ev_join, ss));
  DecryptArgs dca = decrypt_args(c, ct, reinterpret_cast<const int8_t *>(sk), nullptr);
  LAUNCH(c, KID_DECRYPT, st, launch_decrypt(dca, count, st));
  DeriveArgs da = derive_args(c, nullptr, pkh, count);
  LAUNCH(c, KID_DERIVE, st, launch_derive(da, warp_hash_max(c), st));
  rc = run_encrypt(c, pk, A, count, const_cast<uint8_t *>(ct), true, st, nullptr, limbs_from);
  if (rc) return rc;
  CUDA_TRY(cudaStreamWaitEvent(st, c->ev_join, 0));
  final_key(c, z, nullptr, 0, count, K, st);
  return check_launch();
}

int lwe_encaps_multi(lwe_ctx *c, const uint8_t *const *pk_ptrs, const uint8_t *const *pkh_ptrs,
                     const uint16_t *const *A_ptrs, const uint8_t *coins, uint32_t count,
                     uint8_t *ct, uint8_t *K, void *stream) {
  LWE_TRACE("lwe_encaps_multi");
  if (!c) return LWE_EINVAL;
  if (count == 0) return LWE_OK;
  if (count > c->max_batch) return LWE_ECAPACITY;
  if (!pk_ptrs || !coins || !ct || !K || !aligned16(coins) || !aligned16(ct) || !aligned16(K) ||
      (reinterpret_cast<uintptr_t>(pk_ptrs) & 7) || (reinterpret_cast<uintptr_t>(pkh_ptrs) & 7) ||
      (reinterpret_cast<uintptr_t>(A_ptrs) & 7))
    return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_params &p = c->p;
  const size_t pkb = pk_bytes(p), ctb = ct_bytes(p);
  DeriveArgs da = derive_args(c, coins, nullptr, count);
  if (pkh_ptrs) {
    da.pkh_ptrs = pkh_ptrs;
  } else {  // H(pk) of every item's key
    tree_hash(c, nullptr, 0, (uint32_t)pkb, count, TREE_DIGEST, c->pkhs, 32, nullptr, 0, st,
              pk_ptrs);
    da.pkh = c->pkhs;
    da.pkh_stride = 32;
  }
  LAUNCH(c, KID_DERIVE, st, launch_derive(da, warp_hash_max(c), st));
  ItemKeys ik;
  ik.ptrs = pk_ptrs;
  ik.pk_off = 0;
  ik.A_ptrs = A_ptrs;
  rc = run_encrypt(c, nullptr, nullptr, count, ct, false, st, &ik);
  if (rc) return rc;
  return hash_tree(c, ct, ctb, (uint32_t)ctb, count, TREE_ENC_KEY, K, 32, nullptr, 0, st);
}

int lwe_decaps_multi(lwe_ctx *c, const uint8_t *const *sk_ptrs, const uint16_t *const *A_ptrs,
                     const uint8_t *ct, uint32_t count, uint8_t *K, void *stream) {
  LWE_TRACE("lwe_decaps_multi");
  if (!c) return LWE_EINVAL;
  if (count == 0) return LWE_OK;
  if (count > c->max_batch) return LWE_ECAPACITY;
  if (!sk_ptrs || !ct || !K || !aligned16(ct) || !aligned16(K) ||
      (reinterpret_cast<uintptr_t>(sk_ptrs) & 7) || (reinterpret_cast<uintptr_t>(A_ptrs) & 7))
    return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_params &p = c->p;
  const uint32_t n = p.n;
  const size_t ctb = ct_bytes(p);
  CUDA_TRY(cudaMemsetAsync(c->flags, 0, 4 * (size_t)count, st));
  CUDA_TRY(cudaEventRecord(c->ev_fork, st));
  cudaStream_t ss = side_stream(c, st);
  CUDA_TRY(cudaStreamWaitEvent(ss, c->ev_fork, 0));
  tree_hash(c, ct, ctb, (uint32_t)ctb, count, TREE_DIGEST, c->hc, 32, nullptr, 0, ss);
  CUDA_TRY(cudaEventRecord(c->ev_join, ss));
  DecryptArgs dca = decrypt_args(c, ct, nullptr, sk_ptrs);
  LAUNCH(c, KID_DECRYPT, st, launch_decrypt(dca, count, st));
  DeriveArgs da = derive_args(c, nullptr, nullptr, count);
  da.pkh_ptrs = sk_ptrs;  // H(pk) is stored inside sk
  da.pkh_off = 8ull * n + 32;
  LAUNCH(c, KID_DERIVE, st, launch_derive(da, warp_hash_max(c), st));
  ItemKeys ik;
  ik.ptrs = sk_ptrs;
  ik.pk_off = 8ull * n + 64;  // pk is stored inside sk
  ik.A_ptrs = A_ptrs;
  rc = run_encrypt(c, nullptr, nullptr, count, const_cast<uint8_t *>(ct), true, st, &ik);
  if (rc) return rc;
  CUDA_TRY(cudaStreamWaitEvent(st, c->ev_join, 0));
  final_key(c, nullptr, sk_ptrs, 8ull * n, count, K, st);
  return check_launch();
}

int lwe_ctx_bind_key(lwe_ctx *c, const uint8_t *pk, const uint8_t *sk, const uint16_t *A,
                     void *stream) {
  LWE_TRACE("lwe_ctx_bind_key");
  if (!c) return LWE_EINVAL;
  if (!pk && !sk) {
    c->bound = false;
    c->bound_pk = c->bound_sk = nullptr;
    c->bound_A = nullptr;
    return LWE_OK;
  }
  if ((pk && !aligned16(pk)) || (sk && !aligned16(sk)) || (A && !aligned16(A))) return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_params &p = c->p;
  const size_t pkb = pk_bytes(p);
  c->bound = false;
  // pk of the pair: the given one, else the copy inside sk
  const uint8_t *key_pk = pk ? pk : sk + 8 * (size_t)p.n + 64;
  rc = hash_tree(c, key_pk, pkb, (uint32_t)pkb, 1, TREE_DIGEST, c->bpkh, 32, nullptr, 0, st);
  if (rc) return rc;
  if (c->has_tensor) {
    launch_limbs(c, key_pk, A, st, true);
    rc = check_launch();
    if (rc) return rc;
  }
  c->bound = true;
  c->bound_pk = pk;
  c->bound_sk = sk;
  c->bound_A = A;
  return LWE_OK;
}

int lwe_expand_A(const uint8_t *seedA, uint32_t n, uint32_t logq, uint16_t *A_out,
                 void *stream) {
  LWE_TRACE("lwe_expand_A");
  if (!seedA || !A_out || !aligned16(A_out) || n < 16 || n > 65536 || (n % 16) || logq < 1 ||
      logq > 16)
    return LWE_EINVAL;
  int sms = 0;
  int rc = current_device_setup(nullptr, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  launch_expand_A(seedA, 16, 1, n, logq, A_out, 0, sms, st);
  return check_launch();
}

int lwe_matmul_modq(lwe_ctx *c, int side, const uint16_t *A, const uint8_t *seedA,
                    const int8_t *S, uint32_t n, uint32_t k, uint32_t logq, const int8_t *E,
                    uint16_t *out, void *stream) {
  LWE_TRACE("lwe_matmul_modq");
  if (!S || !out || (!A && !seedA) || n < 16 || n > 65536 || (n % 16) || logq < 1 || logq > 16)
    return LWE_EINVAL;
  if (!aligned16(S) || !aligned16(out) || (A && !aligned16(A)) || (E && !aligned16(E)))
    return LWE_EINVAL;
  int sms = 0;
  int rc = current_device_setup(nullptr, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (side == LWE_SIDE_AS) {
    if (k != 8) return LWE_EINVAL;
    MulAsArgs ma;
    memset(&ma, 0, sizeof ma);
    ma.A = A;
    ma.seeds = seedA;
    ma.seed_stride = 16;
    ma.n = n;
    ma.logq = logq;
    ma.St = S;
    ma.E = E;
    ma.out = reinterpret_cast<uint8_t *>(out);
    LAUNCH(c, KID_MUL_AS, st, launch_mul_as(ma, 1, A == nullptr, sms, st));
    return check_launch();
  }
  if (side != LWE_SIDE_SA || k == 0 || (k % 8)) return LWE_EINVAL;
  const uint32_t items = k / 8;
  if (c && c->has_tensor && c->p.n == n && c->p.logq == logq && items <= c->max_batch &&
      (c->path == LWE_PATH_TENSOR ||
       (c->path == LWE_PATH_AUTO && (int)items >= c->tensor_min))) {
    rc = set_device_of(c);
    if (rc) return rc;
    // S and E go through the GEMM as given: convert S to bf16 in the workspace
    GemmLimbArgs la;
    la.A = A;
    la.seedA = seedA;
    la.B = nullptr;
    la.n = n;
    la.logq = logq;
    la.limbs = c->limbs;
    c->limbs_bound = false;  // the bound key's limbs are overwritten
    LAUNCH(c, KID_LIMBS, st, launch_gemm_limbs(la, c->num_sms, st));
    LAUNCH(c, KID_LIMBS, st, launch_s_to_bf16(S, (uint64_t)k * n, c->spbf, c->num_sms, st));
    GemmSaArgs ga;
    memset(&ga, 0, sizeof ga);
    ga.S = c->spbf;
    ga.limbs = c->limbs;
    ga.E = E;
    ga.out = reinterpret_cast<uint8_t *>(out);
    ga.out_stride = 16ull * n;
    ga.dev_err = c->dev_err;
    ga.n = n;
    ga.ncols = n;
    ga.rows = k;
    ga.logq = logq;
    ga.B = 0;
    ga.cmp = 0;
    ga.bn = c->gemm_bn;
    ga.pair = c->gemm_pair;
    ga.group_m = c->gemm_group;
    ga.clip = c->p.clip;
    ga.kchunk = c->kchunk;
    ga.partial_out = c->partial;
    LAUNCH(c, KID_GEMM, st, rc = launch_gemm_sa(ga, c->num_sms, st));
    if (rc) return rc;
    return check_launch();
  }
  MulSaArgs sa;
  memset(&sa, 0, sizeof sa);
  sa.A = A;
  sa.seedA = seedA;
  sa.n = n;
  sa.logq = logq;
  sa.S = S;
  sa.s_stride = 8ull * n;
  sa.E = E;
  sa.e_stride = 8ull * n;
  sa.out = reinterpret_cast<uint8_t *>(out);
  sa.out_stride = 16ull * n;
  LAUNCH(c, A ? KID_MUL_SA : KID_MUL_SA_FUSED, st, launch_mul_sa(sa, items, A == nullptr, false, sms, st));
  return check_launch();
}

int lwe_matmul_modq_rows(int side, const uint16_t *A_rows, const uint8_t *seedA,
                         const int8_t *S, uint32_t n, uint32_t k, uint32_t logq, uint32_t row0,
                         uint32_t row1, const int8_t *E, uint16_t *out, void *stream) {
  LWE_TRACE("lwe_matmul_modq_rows");
  if (!S || !out || (!A_rows && !seedA) || n < 16 || n > 65536 || (n % 16) || logq < 1 ||
      logq > 16)
    return LWE_EINVAL;
  if (row0 >= row1 || row1 > n || (row0 % 16) || (row1 % 16)) return LWE_EINVAL;
  if (!aligned16(S) || !aligned16(out) || (A_rows && !aligned16(A_rows)) || (E && !aligned16(E)))
    return LWE_EINVAL;
  int sms = 0;
  int rc = current_device_setup(nullptr, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (side == LWE_SIDE_AS) {
    if (k != 8) return LWE_EINVAL;
    MulAsArgs ma;
    memset(&ma, 0, sizeof ma);
    ma.A = A_rows;
    ma.seeds = seedA;
    ma.seed_stride = 16;
    ma.n = n;
    ma.logq = logq;
    ma.row0 = row0;
    ma.rows = row1 - row0;
    ma.St = S;
    ma.E = E;
    ma.out = reinterpret_cast<uint8_t *>(out);
    LAUNCH(nullptr, KID_MUL_AS, st, launch_mul_as(ma, 1, A_rows == nullptr, sms, st));
    return check_launch();
  }
  if (side != LWE_SIDE_SA || k == 0 || (k % 8)) return LWE_EINVAL;
  MulSaArgs sa;
  memset(&sa, 0, sizeof sa);
  sa.A = A_rows;
  sa.seedA = seedA;
  sa.n = n;
  sa.logq = logq;
  sa.S = S;
  sa.s_stride = 8ull * n;
  sa.E = E;
  sa.e_stride = 8ull * n;
  sa.out = reinterpret_cast<uint8_t *>(out);
  sa.out_stride = 16ull * n;
  sa.row0 = row0;
  sa.row1 = row1;
  LAUNCH(nullptr, A_rows ? KID_MUL_SA : KID_MUL_SA_FUSED, st,
         launch_mul_sa(sa, k / 8, A_rows == nullptr, false, sms, st));
  return check_launch();
}

int lwe_encaps_noalloc(const lwe_params *p, const uint8_t *pk, const uint16_t *A,
                       const uint8_t *coins, uint32_t count, uint8_t *ct, uint8_t *K,
                       void *stream) {
  LWE_TRACE("lwe_encaps_noalloc");
  if (params_check(p) != LWE_OK) return LWE_EINVAL;
  if (count == 0) return LWE_OK;
  if (!pk || !coins || !ct || !K || !aligned16(pk) || !aligned16(coins) || !aligned16(ct) ||
      !aligned16(K) || (A && !aligned16(A)))
    return LWE_EINVAL;
  const size_t n = p->n, Bm = count;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_seeds = carve(32 * Bm), o_mu = carve(32 * Bm), o_kp = carve(32 * Bm);
  const size_t o_flags = carve(4 * Bm), o_pkh = carve(32), o_rk = carve(176 * Bm);
  const size_t o_sp8 = carve(8 * n * Bm), o_ep8 = carve(8 * n * Bm), o_epp = carve(64 * Bm);
  if (off > LWE_NOALLOC_SCRATCH_BYTES) return LWE_ECAPACITY;

  int dev = 0, sms = 0;
  int rc = current_device_setup(&dev, &sms);
  if (rc) return rc;
  uint8_t *ws = nullptr;
  rc = noalloc_scratch(dev, &ws);
  if (rc) return rc;

  // a context that borrows the built-in scratch instead of owning memory
  lwe_ctx c;
  c.p = *p;
  cdf_table(p->sigma, p->clip, c.T);
  c.device = dev;
  c.num_sms = sms;
  c.max_batch = count;
  c.path = LWE_PATH_SKINNY;
  c.has_tensor = false;
  c.seeds = ws + o_seeds;
  c.mu = ws + o_mu;
  c.kp = ws + o_kp;
  c.flags = reinterpret_cast<uint32_t *>(ws + o_flags);
  c.rk = reinterpret_cast<uint32_t *>(ws + o_rk);
  c.pkh = ws + o_pkh;
  c.sp8 = reinterpret_cast<int8_t *>(ws + o_sp8);
  c.ep8 = reinterpret_cast<int8_t *>(ws + o_ep8);
  c.epp = reinterpret_cast<int8_t *>(ws + o_epp);

  cudaStream_t st = (cudaStream_t)stream;
  const size_t pkb = pk_bytes(*p), ctb = ct_bytes(*p);
  rc = hash_tree(&c, pk, pkb, (uint32_t)pkb, 1, TREE_DIGEST, c.pkh, 32, nullptr, 0, st);
  if (rc) return rc;
  DeriveArgs da = derive_args(&c, coins, c.pkh, count);
  LAUNCH(&c, KID_DERIVE, st, launch_derive(da, warp_hash_max(&c), st));
  rc = run_encrypt(&c, pk, A, count, ct, false, st);
  if (rc) return rc;
  return hash_tree(&c, ct, ctb, (uint32_t)ctb, count, TREE_ENC_KEY, K, 32, nullptr, 0, st);
}

int lwe_noise_table(const lwe_params *p, int8_t *out, void *stream) {
  LWE_TRACE("lwe_noise_table");
  if (params_check(p) != LWE_OK || !out) return LWE_EINVAL;
  int rc = current_device_setup(nullptr, nullptr);
  if (rc) return rc;
  NoiseArgs a;
  memset(&a, 0, sizeof a);
  uint16_t T[16];
  cdf_table(p->sigma, p->clip, T);
  for (int i = 0; i < 16; i++) a.T[i] = T[i];
  launch_noise_table(a, out, (cudaStream_t)stream);
  return check_launch();
}

int lwe_bounds_violations(uint64_t *count, uint32_t *first_site) {
#ifndef LWE_CHECK_BOUNDS
  (void)count;
  (void)first_site;
  return LWE_EUNSUPPORTED;
#else
  if (!count || !first_site) return LWE_EINVAL;
  CUDA_TRY(cudaDeviceSynchronize());
  unsigned long long c1 = 0, c2 = 0;
  unsigned s1 = 0, s2 = 0;
  CUDA_TRY(lwe_bounds_read_kem(&c1, &s1));
  CUDA_TRY(lwe_bounds_read_gemm(&c2, &s2));
  *count = c1 + c2;
  *first_site = c1 ? s1 : (c2 ? s2 : 0);
  return LWE_OK;
#endif
}

int lwe_probe(int kind, uint32_t ctas, uint32_t iters, uint32_t *sink, void *stream) {
  if (kind < LWE_PROBE_KECCAK || kind > LWE_PROBE_AES_RUN || ctas == 0 || !sink ||
      (kind == LWE_PROBE_AES && (iters & 1)) ||
      (kind == LWE_PROBE_AES_RUN && (iters % (NOISE_RUN / 32))))
    return LWE_EINVAL;
  int rc = current_device_setup(nullptr, nullptr);
  if (rc) return rc;
  launch_probe(kind, ctas, iters, sink, (cudaStream_t)stream);
  return check_launch();
}

int lwe_selftest_bounded_wait(lwe_ctx *c, uint32_t limit_us, void *stream) {
  if (!c || limit_us == 0 || limit_us > 2000000) return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  launch_selftest_wait(c->dev_err, (uint64_t)limit_us * 1000ull, (cudaStream_t)stream);
  return check_launch();
}

const char *lwe_strerror(int code) {
  switch (code) {
    case LWE_OK: return "ok";
    case LWE_EINVAL: return "invalid argument";
    case LWE_ENOMEM: return "out of device memory";
    case LWE_ECUDA: return "CUDA error";
    case LWE_ETIMEOUT: return "device wait timed out";
    case LWE_EUNSUPPORTED: return "unsupported device or configuration";
    case LWE_ECAPACITY:
      return "count exceeds the context's max_batch or the built-in scratch area";
    default: return "unknown error";
  }
}

const char *lwe_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int lwe_ctx_device_error(lwe_ctx *c) {
  if (!c) return LWE_EINVAL;
  int rc = set_device_of(c);
  if (rc) return rc;
  CUDA_TRY(cudaDeviceSynchronize());
  uint32_t v = 0;
  CUDA_TRY(cudaMemcpy(&v, c->dev_err, 4, cudaMemcpyDeviceToHost));
  if (v) {
    CUDA_TRY(cudaMemset(c->dev_err, 0, 4));
    return LWE_ETIMEOUT;
  }
  return LWE_OK;
}

uint64_t lwe_ctx_launches(const lwe_ctx *c) { return c ? c->launches : 0; }

int lwe_ctx_kernel_stats(lwe_ctx *c, int kid, uint64_t *launches, double *total_ms) {
  if (!c || kid < 0 || kid >= KID_COUNT) return LWE_EINVAL;
  harvest(c);
  if (launches) *launches = c->stat_launches[kid];
  if (total_ms) *total_ms = c->stat_ms[kid];
  return LWE_OK;
}

int lwe_ctx_timing_mark(lwe_ctx *c) {
  if (!c) return LWE_EINVAL;
  for (auto &t : c->replay) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  c->replay.swap(c->pending);
  c->pending.clear();
  return LWE_OK;
}

int lwe_ctx_timing_replay(lwe_ctx *c) {
  if (!c) return LWE_EINVAL;
  for (auto &t : c->replay) {
    CUDA_TRY(cudaEventSynchronize(t.b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, t.a, t.b));
    c->stat_launches[t.kid]++;
    c->stat_ms[t.kid] += ms;
  }
  return LWE_OK;
}

int lwe_ctx_reset_stats(lwe_ctx *c) {
  if (!c) return LWE_EINVAL;
  harvest(c);
  for (int i = 0; i < KID_COUNT; i++) {
    c->stat_launches[i] = 0;
    c->stat_ms[i] = 0.0;
  }
  return LWE_OK;
}

const char *lwe_kernel_name(int kid) {
  if (kid < 0 || kid >= KID_COUNT) return nullptr;
  return kKernelNames[kid];
}

int lwe_num_kernels(void) { return KID_COUNT; }

}  // extern "C"

// ===========================================================================
// The paper's own parameter profile (lwe_pp.h; Tab. 1, Alg. 1-5 with odd q
// and a 256-bit message encrypted bit by bit)
// ===========================================================================
namespace {

// Tab. 1: n, q, sigma, k; the clip is the largest (<= 15) whose CDF table is
// valid for that sigma
const struct {
  uint32_t n, q;
  double sigma;
  uint32_t k;
} kPpPresets[] = {{512, 3329, 2.3, 3},   {1024, 12289, 2.3, 3}, {2048, 12289, 2.3, 3},
                  {4096, 12289, 1.7, 3}, {8192, 65537, 1.2, 2}, {16384, 65537, 1.2, 2},
                  {32768, 65537, 1.0, 2}};

ModQ modq(uint32_t q) { return ModQ{q, (uint32_t)(0x100000000ull / q)}; }

size_t pp_pk_bytes(const lwe_pp_params &p) { return 16 + 4 * (size_t)p.n; }
size_t pp_sk_bytes(const lwe_pp_params &p) { return p.n + 64 + pp_pk_bytes(p); }
size_t pp_ct_bytes(const lwe_pp_params &p) { return 4 * (size_t)PP_MBITS * p.n + 4 * PP_MBITS; }

}  // namespace

struct lwe_pp_ctx {
  lwe_pp_params p;
  uint16_t T[16];
  int device = 0, num_sms = 0;
  uint8_t *ws = nullptr;
  uint8_t *seeds = nullptr, *mu = nullptr, *kp = nullptr, *pkh = nullptr, *hc = nullptr;
  uint8_t *digests = nullptr;  // 257 x 32: the rows' and v's tree hashes
  uint32_t *rk = nullptr, *flags = nullptr;
  int8_t *e = nullptr, *Rt = nullptr, *E1t = nullptr;
  int32_t *e2 = nullptr;
  uint32_t *dev_err = nullptr;
  uint16_t *Rbf = nullptr;     // r^T as bf16 (GEMM operand)
  uint16_t *limbs = nullptr;   // [2][n][n] bf16 limbs of A
  uint32_t *partial = nullptr; // K-split running sums, [256][n] mod q
  bool tensor = false;         // LWE_PP_OPT_TENSOR (set when the GEMM supports n)
  bool pdl = false;            // LWE_PP_OPT_PDL
  // the key bound by lwe_pp_ctx_bind_key: its pk and A buffers, H(pk)
  // (bpkh), and whether `limbs` still holds the limbs of its A
  const uint8_t *bound_pk = nullptr;
  const uint32_t *bound_A = nullptr;
  uint8_t *bpkh = nullptr;
  bool limbs_bound = false;
};

namespace {

void pp_tree(lwe_pp_ctx *c, const uint8_t *msgs, uint64_t stride, uint32_t len, uint32_t count,
             int mode, uint8_t *out, uint64_t out_stride, cudaStream_t st) {
  TreeArgs ta;
  memset(&ta, 0, sizeof ta);
  ta.msgs = msgs;
  ta.stride = stride;
  ta.len = len;
  ta.count = count;
  ta.mode = mode;
  ta.out = out;
  ta.out_stride = out_stride;
  ta.kprime = c->kp;
  launch_tree(ta, c->num_sms, (uint32_t)c->num_sms, st);
}

// H(c) = Htree(Htree(u_0) || ... || Htree(u_255) || Htree(v)); with
// TREE_ENC_KEY the last launch returns K = H(K' || H(c)) instead
void pp_hash_ct(lwe_pp_ctx *c, const uint8_t *ct, int mode, uint8_t *out, cudaStream_t st) {
  const uint32_t row = 4 * c->p.n;
  pp_tree(c, ct, row, row, PP_MBITS, TREE_DIGEST, c->digests, 32, st);
  pp_tree(c, ct + (size_t)PP_MBITS * row, 4 * PP_MBITS, 4 * PP_MBITS, 1, TREE_DIGEST,
          c->digests + 32 * PP_MBITS, 32, st);
  pp_tree(c, c->digests, 32 * (PP_MBITS + 1), 32 * (PP_MBITS + 1), 1, mode, out, 32, st);
}

// Encrypt's noise from the round keys in c->rk: r, e1 (Gaussian, 256 x n)
// and e2 (centred uniform, 256)
void pp_encrypt_noise(lwe_pp_ctx *c, cudaStream_t st) {
  PpNoiseArgs na;
  memset(&na, 0, sizeof na);
  na.rk = c->rk;
  const uint32_t n = c->p.n;
  na.o[0] = PpNoiseOut{c->Rt, PP_MBITS * n, PP_GAUSS, 3, 0};
  na.o[1] = PpNoiseOut{c->E1t, PP_MBITS * n, PP_GAUSS, 4, 0};
  na.o[2] = PpNoiseOut{c->e2, PP_MBITS, PP_UNIFORM, 5, 0};
  na.nout = 3;
  na.clip = c->p.clip;
  na.kunif = c->p.k;
  for (int i = 0; i < 16; i++) na.T[i] = c->T[i];
  launch_pp_noise(na, c->num_sms, st);
}

// U^T and v of Encrypt from c's noise and message c->mu; cmp compares them
// with ct (Decaps) instead of writing
int pp_encrypt(lwe_pp_ctx *c, const uint32_t *t, const uint32_t *A, uint8_t *ct, bool cmp,
               cudaStream_t st) {
  const uint32_t n = c->p.n;
  const ModQ M = modq(c->p.q);
  if (c->tensor) {
    // U^T = R^T A + E1^T on the tensor cores; the bound key's limbs are
    // made once
    if (!(A == c->bound_A && c->limbs_bound)) {
      launch_pp_limbs(A, n, c->p.q, c->limbs, st);
      c->limbs_bound = A == c->bound_A;
    }
    launch_s_to_bf16(c->Rt, (uint64_t)PP_MBITS * n, c->Rbf, c->num_sms, st);
    GemmSaArgs ga;
    memset(&ga, 0, sizeof ga);
    ga.S = c->Rbf;
    ga.limbs = c->limbs;
    ga.E = c->E1t;
    ga.out = ct;
    ga.flags = c->flags;
    ga.dev_err = c->dev_err;
    ga.n = n;
    ga.ncols = n;
    ga.rows = PP_MBITS;
    ga.logq = 16;
    ga.cmp = cmp ? 1 : 0;
    ga.bn = 128;
    ga.pair = 1;
    ga.clip = c->p.clip;
    ga.kchunk = lwe_gemm_kchunk(c->p.clip);
    ga.partial_out = reinterpret_cast<uint16_t *>(c->partial);
    ga.oddq_q = M.q;
    ga.oddq_m = M.m;
    const int rc = launch_gemm_sa(ga, c->num_sms, st);
    if (rc != LWE_OK) return rc;
  } else {
    PpEncArgs ea{A, c->Rt, c->E1t, reinterpret_cast<uint32_t *>(ct), c->flags, n, M};
    launch_pp_encrypt(ea, cmp, st);
  }
  PpVArgs va{t, c->Rt, c->e2, c->mu, reinterpret_cast<uint32_t *>(ct) + (size_t)PP_MBITS * n,
             c->flags, n, M};
  launch_pp_v(va, cmp, st);
  return LWE_OK;
}

// programmatic dependent launch for the paper-profile calls when enabled
// (every kernel they use waits on the device for its predecessor)
struct PdlOn {
  bool before = g_launch_pdl;
  explicit PdlOn(bool on) { g_launch_pdl = on; }
  ~PdlOn() { g_launch_pdl = before; }
};

DeriveArgs pp_derive_args(lwe_pp_ctx *c, const uint8_t *coins, const uint8_t *pkh) {
  DeriveArgs da;
  memset(&da, 0, sizeof da);
  da.coins = coins;
  da.pkh = pkh;
  da.pkh_stride = 32;
  da.mu = c->mu;
  da.kprime = c->kp;
  da.seeds = c->seeds;
  da.rk = c->rk;
  da.count = 1;
  da.mu_bytes = 32;
  return da;
}

}  // namespace

extern "C" {

int lwe_pp_params_preset(int id, lwe_pp_params *out) {
  if (!out || id < 0 || id >= (int)(sizeof kPpPresets / sizeof kPpPresets[0])) return LWE_EINVAL;
  lwe_pp_params p;
  p.n = kPpPresets[id].n;
  p.q = kPpPresets[id].q;
  p.sigma = kPpPresets[id].sigma;
  p.k = kPpPresets[id].k;
  uint16_t T[16];
  p.clip = 15;
  while (p.clip > 1 && cdf_table(p.sigma, p.clip, T) != LWE_OK) p.clip--;
  *out = p;
  return LWE_OK;
}

int lwe_pp_params_check(const lwe_pp_params *p) {
  if (!p) return LWE_EINVAL;
  if (p->n < 64 || p->n > 65536 || (p->n % 64)) return LWE_EINVAL;
  if (p->q < 3 || p->q > 65537 || !(p->q & 1)) return LWE_EINVAL;
  if (p->k < 1 || p->k > 15) return LWE_EINVAL;
  uint16_t T[16];
  return cdf_table(p->sigma, p->clip, T);
}

size_t lwe_pp_pk_bytes(const lwe_pp_params *p) { return p ? pp_pk_bytes(*p) : 0; }
size_t lwe_pp_sk_bytes(const lwe_pp_params *p) { return p ? pp_sk_bytes(*p) : 0; }
size_t lwe_pp_ct_bytes(const lwe_pp_params *p) { return p ? pp_ct_bytes(*p) : 0; }

int lwe_pp_ctx_create(const lwe_pp_params *p, int device, lwe_pp_ctx **out) {
  if (!out) return LWE_EINVAL;
  *out = nullptr;
  if (lwe_pp_params_check(p) != LWE_OK) return LWE_EINVAL;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return LWE_EINVAL;
  int rc = device_setup(device);
  if (rc != LWE_OK) return rc;
  int prev = 0;
  CUDA_TRY(cudaGetDevice(&prev));
  CUDA_TRY(cudaSetDevice(device));
  lwe_pp_ctx *c = new lwe_pp_ctx();
  c->p = *p;
  cdf_table(p->sigma, p->clip, c->T);
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  const size_t n = p->n;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_seeds = carve(32), o_mu = carve(32), o_kp = carve(32), o_pkh = carve(32);
  const size_t o_bpkh = carve(32);
  const size_t o_hc = carve(32), o_dig = carve(32 * (PP_MBITS + 1)), o_rk = carve(176);
  const size_t o_flags = carve(16), o_e = carve(n), o_Rt = carve(PP_MBITS * n);
  const size_t o_E1t = carve(PP_MBITS * n), o_e2 = carve(4 * PP_MBITS), o_err = carve(16);
  const bool tensor = lwe_gemm_supported((uint32_t)n, 16, p->clip);
  size_t o_Rbf = 0, o_limbs = 0, o_partial = 0;
  if (tensor) {
    o_Rbf = carve(2 * PP_MBITS * n);
    o_limbs = carve(4 * n * n);
    o_partial = carve(4 * PP_MBITS * n);
  }
  cudaError_t e = cudaMalloc(&c->ws, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    cudaSetDevice(prev);
    return LWE_ENOMEM;
  }
  c->seeds = c->ws + o_seeds;
  c->mu = c->ws + o_mu;
  c->kp = c->ws + o_kp;
  c->pkh = c->ws + o_pkh;
  c->bpkh = c->ws + o_bpkh;
  c->hc = c->ws + o_hc;
  c->digests = c->ws + o_dig;
  c->rk = reinterpret_cast<uint32_t *>(c->ws + o_rk);
  c->flags = reinterpret_cast<uint32_t *>(c->ws + o_flags);
  c->e = reinterpret_cast<int8_t *>(c->ws + o_e);
  c->Rt = reinterpret_cast<int8_t *>(c->ws + o_Rt);
  c->E1t = reinterpret_cast<int8_t *>(c->ws + o_E1t);
  c->e2 = reinterpret_cast<int32_t *>(c->ws + o_e2);
  c->dev_err = reinterpret_cast<uint32_t *>(c->ws + o_err);
  c->tensor = tensor;
  if (tensor) {
    c->Rbf = reinterpret_cast<uint16_t *>(c->ws + o_Rbf);
    c->limbs = reinterpret_cast<uint16_t *>(c->ws + o_limbs);
    c->partial = reinterpret_cast<uint32_t *>(c->ws + o_partial);
  }
  e = cudaMemset(c->ws, 0, off);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return cuda_fail(e);
  }
  *out = c;
  return LWE_OK;
}

int lwe_pp_ctx_destroy(lwe_pp_ctx *c) {
  if (!c) return LWE_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->ws);
  cudaSetDevice(prev);
  delete c;
  return LWE_OK;
}

int lwe_pp_ctx_set_option(lwe_pp_ctx *c, int option, int64_t value) {
  if (!c) return LWE_EINVAL;
  if (value != 0 && value != 1) return LWE_EINVAL;
  if (option == LWE_PP_OPT_TENSOR) {
    if (value && !c->limbs) return LWE_EUNSUPPORTED;
    c->tensor = value != 0;
    return LWE_OK;
  }
  if (option == LWE_PP_OPT_PDL) {
    c->pdl = value != 0;
    return LWE_OK;
  }
  return LWE_EINVAL;
}

int lwe_pp_expand_A(const lwe_pp_params *p, const uint8_t *seedA, uint32_t *A, void *stream) {
  LWE_TRACE("lwe_pp_expand_A");
  if (lwe_pp_params_check(p) != LWE_OK || !seedA || !A || !aligned16(A)) return LWE_EINVAL;
  int sms = 0;
  int rc = current_device_setup(nullptr, &sms);
  if (rc) return rc;
  launch_pp_expand_A(seedA, p->n, modq(p->q), A, sms, (cudaStream_t)stream);
  return check_launch();
}

int lwe_pp_keygen(lwe_pp_ctx *c, const uint8_t *seed32, uint8_t *pk, uint8_t *sk, uint32_t *A,
                  void *stream) {
  LWE_TRACE("lwe_pp_keygen");
  if (!c || !seed32 || !pk || !sk || !A || !aligned16(pk) || !aligned16(sk) || !aligned16(A))
    return LWE_EINVAL;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_pp_params &p = c->p;
  const uint32_t n = p.n;
  const ModQ M = modq(p.q);
  PdlOn pdl(c->pdl);
  // seedA -> pk, the copy of pk in sk and seeds[0:16]; seedSE -> seeds[16:32]
  // and its key schedule; z -> sk
  KeygenSeedArgs ka;
  memset(&ka, 0, sizeof ka);
  ka.ms = seed32;
  ka.pk = pk;
  ka.sk = sk;
  ka.ws_seeds = c->seeds;
  ka.ws_rk = c->rk;
  ka.pk_bytes = pp_pk_bytes(p);
  ka.sk_bytes = pp_sk_bytes(p);
  ka.sk_z_off = n;
  ka.sk_pk_off = n + 64;
  ka.count = 1;
  launch_keygen_seeds(ka, (uint32_t)c->num_sms, st);
  launch_pp_expand_A(c->seeds, n, M, A, c->num_sms, st);
  PpNoiseArgs na;
  memset(&na, 0, sizeof na);
  na.rk = c->rk;
  na.o[0] = PpNoiseOut{sk, n, PP_BINOMIAL, 1, 0};  // s: the first n bytes of sk
  na.o[1] = PpNoiseOut{c->e, n, PP_GAUSS, 2, 0};
  na.nout = 2;
  na.clip = p.clip;
  na.kunif = p.k;
  for (int i = 0; i < 16; i++) na.T[i] = c->T[i];
  launch_pp_noise(na, c->num_sms, st);
  PpAsArgs aa{A, reinterpret_cast<const int8_t *>(sk), c->e, reinterpret_cast<uint32_t *>(pk + 16),
              reinterpret_cast<uint32_t *>(sk + n + 64 + 16), n, M};
  launch_pp_as(aa, st);
  pp_tree(c, pk, pp_pk_bytes(p), (uint32_t)pp_pk_bytes(p), 1, TREE_DIGEST, sk + n + 32, 32, st);
  return check_launch();
}

int lwe_pp_encaps(lwe_pp_ctx *c, const uint8_t *pk, const uint32_t *A, const uint8_t *coins32,
                  uint8_t *ct, uint8_t *K, void *stream) {
  LWE_TRACE("lwe_pp_encaps");
  if (!c || !pk || !A || !coins32 || !ct || !K || !aligned16(pk) || !aligned16(A) ||
      !aligned16(ct))
    return LWE_EINVAL;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_pp_params &p = c->p;
  PdlOn pdl(c->pdl);
  const uint8_t *pkh = c->bpkh;  // the bound key's H(pk), made once
  if (pk != c->bound_pk) {
    pp_tree(c, pk, pp_pk_bytes(p), (uint32_t)pp_pk_bytes(p), 1, TREE_DIGEST, c->pkh, 32, st);
    pkh = c->pkh;
  }
  // m = H(0x4D || coins), K' = H(H(pk) || m), seedSE' and its key schedule
  launch_derive(pp_derive_args(c, coins32, pkh), (uint32_t)c->num_sms, st);
  pp_encrypt_noise(c, st);
  const int rc = pp_encrypt(c, reinterpret_cast<const uint32_t *>(pk + 16), A, ct, false, st);
  if (rc != LWE_OK) return rc;
  pp_hash_ct(c, ct, TREE_ENC_KEY, K, st);  // K = H(K' || H(c))
  return check_launch();
}

int lwe_pp_ctx_bind_key(lwe_pp_ctx *c, const uint8_t *pk, const uint32_t *A, void *stream) {
  LWE_TRACE("lwe_pp_ctx_bind_key");
  if (!c) return LWE_EINVAL;
  c->bound_pk = nullptr;
  c->bound_A = nullptr;
  c->limbs_bound = false;
  if (!pk && !A) return LWE_OK;
  if ((pk && !aligned16(pk)) || (A && !aligned16(A))) return LWE_EINVAL;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_pp_params &p = c->p;
  if (pk) pp_tree(c, pk, pp_pk_bytes(p), (uint32_t)pp_pk_bytes(p), 1, TREE_DIGEST, c->bpkh, 32, st);
  if (A && c->tensor) {
    launch_pp_limbs(A, p.n, p.q, c->limbs, st);
    c->limbs_bound = true;
  }
  const int rc = check_launch();
  if (rc) return rc;
  c->bound_pk = pk;
  c->bound_A = A;
  return LWE_OK;
}

int lwe_pp_decaps(lwe_pp_ctx *c, const uint8_t *sk, const uint32_t *A, const uint8_t *ct,
                  uint8_t *K, void *stream) {
  LWE_TRACE("lwe_pp_decaps");
  if (!c || !sk || !A || !ct || !K || !aligned16(sk) || !aligned16(A) || !aligned16(ct))
    return LWE_EINVAL;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const lwe_pp_params &p = c->p;
  const uint32_t n = p.n;
  const uint8_t *z = sk + n, *pkh = sk + n + 32, *pk = sk + n + 64;
  PdlOn pdl(c->pdl);
  CUDA_TRY(cudaMemsetAsync(c->flags, 0, 4, st));
  CUDA_TRY(cudaMemsetAsync(c->mu, 0, 32, st));
  PpDecArgs dargs{reinterpret_cast<const uint32_t *>(ct),
                  reinterpret_cast<const uint32_t *>(ct) + (size_t)PP_MBITS * n,
                  reinterpret_cast<const int8_t *>(sk), reinterpret_cast<uint32_t *>(c->mu), n,
                  modq(p.q)};
  launch_pp_decrypt(dargs, st);  // m' into c->mu
  launch_derive(pp_derive_args(c, nullptr, pkh), (uint32_t)c->num_sms, st);
  pp_encrypt_noise(c, st);
  const int rc = pp_encrypt(c, reinterpret_cast<const uint32_t *>(pk + 16), A,
                            const_cast<uint8_t *>(ct), true, st);
  if (rc != LWE_OK) return rc;
  pp_hash_ct(c, ct, TREE_DIGEST, c->hc, st);
  FinalKeyArgs fa;
  memset(&fa, 0, sizeof fa);
  fa.kprime = c->kp;
  fa.hc = c->hc;
  fa.z = z;
  fa.flags = c->flags;
  fa.K = K;
  fa.count = 1;
  launch_final_key(fa, (uint32_t)c->num_sms, st);
  return check_launch();
}

}  // extern "C"
