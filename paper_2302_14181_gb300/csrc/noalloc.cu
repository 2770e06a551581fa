// tevo_gemm_noalloc: the complex contraction of tevo_gemm for callers that must
// not allocate device memory -- for example a process that has handed the whole
// device to a pre-sized memory pool, or code running where an allocation could
// block, fail or be forbidden (between operations of a latency-critical service,
// or in a runtime that owns the allocator). Its temporary storage (operand
// planes, split-K partials, the error flag of the bounded waits) lives in one
// file-scope __device__ array, created when the library is loaded and held by
// every GPU that loads it until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "tevo_mixed.h"
#include "tevo_tc.h"

namespace tevo {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TEVO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the context's device (host code may
// not use the symbol itself as an address); looked up once per device, with
// that device current. The context's kernels run on its stream, so a call made
// while another device is current is refused: the address would belong to the
// other device's copy of the array.
int scratch_for_device(int ctx_device, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TEVO_ECUDA;
  if (dev != ctx_device) return TEVO_EINVAL;
  if (dev < 0 || dev >= kMaxDevices) return TEVO_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TEVO_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return 0;
}

inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }
inline long long pad8(long long x) { return (x + 7) / 8 * 8; }

int fmt_of(int precision) {
  return precision == TEVO_TF32 ? TC_TF32 : precision == TEVO_TF32X3 ? TC_TF32X3 : TC_BF16;
}

}  // namespace

#define TRY_NA(x)      \
  do {                 \
    int _e = (x);      \
    if (_e) return _e; \
  } while (0)

// bytes of scratch a call of this shape needs; the layout is
// [error flag | A planes | B planes | split-K partials]. The split-K count is the
// one tevo_gemm would use, lowered until the partials fit the scratch array.
// Returns 0 when the shape cannot fit at all.
size_t noalloc_need(int precision, int M, int N, int K, int num_sms, int* splits_out) {
  const size_t limit = (size_t)TEVO_NOALLOC_SCRATCH_BYTES;
  if (precision == TEVO_FP64) {
    GemmDesc g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.batch = 1;
    *splits_out = 1;
    const size_t ws = zgemm64_workspace(g, num_sms);
    // without room for the split-K partials the fp64 GEMM runs unsplit
    return 256 + (256 + ws <= limit ? ws : 0);
  }
  const int fmt = fmt_of(precision);
  const int P = tc_planes(fmt), eb = tc_elem_bytes(fmt);
  const long long kp = pad8(K);
  const size_t planes = al256((size_t)P * M * kp * eb) + al256((size_t)P * N * kp * eb);
  if (256 + planes + al256((size_t)M * N * 8) > limit) return 0;
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
  const int kc = tc_kchunk(fmt);
  const int ktiles = (K + kc - 1) / kc;
  int splits = std::max(1, std::min({num_sms / std::max(1, tiles), ktiles, 64}));
  const size_t room = (limit - 256 - planes) / ((size_t)M * N * 8 + 256);
  splits = std::max(1, std::min<int>(splits, (int)std::min<size_t>(room, 64)));
  const int tps = (ktiles + splits - 1) / splits;
  splits = (ktiles + tps - 1) / tps;
  *splits_out = splits;
  return 256 + planes + al256((size_t)splits * M * N * 8);
}

int noalloc_gemm(const Launch& L, int device, int precision, int M, int N, int K, const void* A, const void* B,
                 void* C) {
  void* base = nullptr;
  TRY_NA(scratch_for_device(device, &base));
  int splits = 1;
  const size_t need = noalloc_need(precision, M, N, K, L.num_sms, &splits);
  if (need == 0 || need > (size_t)TEVO_NOALLOC_SCRATCH_BYTES) return TEVO_ESHAPE;
  char* p = static_cast<char*>(base);
  int* err = reinterpret_cast<int*>(p);
  // the flag keeps the previous call's value: clear it before any kernel runs
  if (cudaMemsetAsync(err, 0, 256, L.stream) != cudaSuccess) return TEVO_ECUDA;
  p += 256;
  if (precision == TEVO_FP64) {
    GemmDesc g{};
    g.A = A;
    g.B = B;
    g.C = C;
    g.M = M;
    g.N = N;
    g.K = K;
    g.batch = 1;
    g.sAm = K;
    g.sAk = 1;
    g.sBk = 1;
    g.sBn = K;
    g.sCm = N;
    g.sCn = 1;
    g.alpha_re = 1.0;
    TRY_NA(zgemm64(L, g, p, need - 256));
    return cudaStreamSynchronize(L.stream) == cudaSuccess ? 0 : TEVO_ECUDA;
  }
  const int fmt = fmt_of(precision);
  const int P = tc_planes(fmt), eb = tc_elem_bytes(fmt);
  const long long kp = pad8(K);
  void* pa = p;
  p += al256((size_t)P * M * kp * eb);
  void* pb = p;
  p += al256((size_t)P * N * kp * eb);
  float2* part = reinterpret_cast<float2*>(p);
  for (int side = 0; side < 2; ++side) {
    TcConvert cv;
    std::memset(&cv, 0, sizeof(cv));
    cv.src = side == 0 ? A : B;
    cv.rows = side == 0 ? M : N;
    cv.K = K;
    cv.R2 = cv.rows;
    cv.sR2 = K;
    cv.K2 = K;
    cv.sK2 = 1;
    cv.fmt = fmt;
    cv.dst.base = side == 0 ? pa : pb;
    cv.dst.plane_stride = (long long)cv.rows * kp;
    cv.row_pitch = kp;
    cv.kin = K;
    TRY_NA(tc_to_planes(L, cv));
  }
  TcOperand oa{pa, eb, P, (long long)M * kp, M, kp, K, 1, kp};
  TcOperand ob{pb, eb, P, (long long)N * kp, N, kp, K, 1, kp};
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.err = err;
  a.out_mode = TC_OUT_PARTIAL;
  a.splits = splits;
  a.partial = part;
  TRY_NA(tc_gemm(L, fmt, oa, ob, M, N, a));
  TRY_NA(tc_reduce_partials(L, part, splits, M, N, C, N, 1));
  int flag = 0;
  if (cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
      cudaStreamSynchronize(L.stream) != cudaSuccess)
    return TEVO_ECUDA;
  return flag ? TEVO_ETIMEOUT : 0;
}

}  // namespace tevo
