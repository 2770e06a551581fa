// Internal declarations shared by the translation units of libtevo.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/tevo.h"

#ifdef __CUDACC__
#include <cuda_runtime.h>

#include <atomic>
#else
struct CUstream_st;
typedef CUstream_st* cudaStream_t;
#endif

namespace tevo {

// bumped whenever a persistent device buffer of a handle is (re)allocated;
// captured CUDA graphs of the batched form are dropped when it changes
extern long long g_persist_gen;

// host MPO construction (mpo_build.cpp)
int build_mpo_host(int L, int d, int chi, const double* A, const double* B, const double* C,
                   const double* Dh, int N, double tau_re, double tau_im, int variant,
                   std::vector<std::vector<std::complex<double>>>& sites, std::vector<int>& wl,
                   std::vector<int>& wr);

// complex fp64 as two doubles
struct z64 {
  double x, y;
};

// Strided batched complex GEMM description: C[b](m,n) = alpha * sum_k op(A)[b](m,k) op(B)[b](k,n)
// (+ beta * C). Strides are in complex elements; op() conjugates when conj* is set.
struct GemmDesc {
  const void* A;
  const void* B;
  void* C;
  int M, N, K, batch;
  long long sAb, sAm, sAk;
  long long sBb, sBk, sBn;
  long long sCb, sCm, sCn;
  int conjA, conjB;
  double alpha_re, alpha_im, beta_re, beta_im;
};

// event-timed profile of kernel classes (TEVO_PROF_*)
struct Prof {
  bool on = false;
  struct Rec {
    int cls;
    void* e0;
    void* e1;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  std::vector<void*> pool;  // cudaEvent_t
  // returns an index into recs (or -1 when off); the caller launches between begin/end
  int begin(cudaStream_t s, int cls, double flops, double bytes);
  void end(cudaStream_t s, int idx);
};

// launch-side context passed to the kernel wrappers
struct Launch {
  cudaStream_t stream;
  long long* launches;  // incremented per kernel launch
  int num_sms;
  Prof* prof;
};

#ifdef __CUDACC__
// Raise a kernel's dynamic shared-memory limit on the current device. The
// attribute is kept per device, so `done` holds one bit per device (devices
// 0..63; higher ones set it on every call). Concurrent first calls may both set
// it, which is harmless.
template <typename F>
inline int smem_attr_once(F* kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TEVO_ECUDA;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return 0;
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes) != cudaSuccess)
    return TEVO_ECUDA;
  done.fetch_or(bit, std::memory_order_release);
  return 0;
}
#endif

// ---------------------------------------------------------------------------
// fp64 kernels (k_fp64.cu)
// ---------------------------------------------------------------------------
// workspace bytes needed by zgemm64 for this description (split-K partials)
size_t zgemm64_workspace(const GemmDesc& g, int num_sms);
int zgemm64(const Launch& L, const GemmDesc& g, void* workspace, size_t ws_bytes);

// fp64 complex GEMM on the bf16 tensor cores by the Ozaki splitting scheme
// (k_oz.cu): batch 1, alpha 1, beta 0, conjB 0 only (else TEVO_EUNSUPPORTED);
// slices in 1..oz_max_slices(). A device wait that gives up sets *err (never
// cleared here).
int oz_max_slices();
size_t ozgemm64_workspace(const GemmDesc& g, int slices, int num_sms);
int ozgemm64(const Launch& L, const GemmDesc& g, int slices, void* ws, size_t ws_bytes, int* err);

// G2 over the nonzeros of the MPO operand (CSR rows of [(s v)][(wl s')]):
// T[p][r][b] = sum_k W[r][k] X[p][k][b], batch p, R rows, K = wl d, Db columns
int zsparse_g2(const Launch& L, const z64* X, z64* T, const int* row_ptr, const int* col_idx, const z64* vals,
               int R, int K, int Db, int batch);

// Householder QR of a column-major m x n matrix (ld = m), in place.
// V (m x n col-major) receives the reflectors, tau/beta (n) the scalars.
// scratch: >= qr64_scratch_bytes(m, n).
size_t qr64_scratch_bytes(int m, int n);
int qr64_factor(const Launch& L, z64* A, int m, int n, z64* V, z64* tau, z64* beta, void* scratch);
// the same factorisation as one cooperative launch (columns owned by CTAs, the
// reflectors passed through V with release/acquire flags[k] = epoch); returns
// TEVO_EUNSUPPORTED when the matrix does not fit (then use qr64_factor)
int qr64_factor_coop(const Launch& L, z64* A, int m, int n, z64* V, z64* tau, z64* beta, void* scratch, int* flags,
                     int epoch, int* err);
// explicit thin Q (m x n) written with element (r, c) at Q[r * sQr + c * sQc],
// from the compact WY form of blocks of reflectors; wy: qr64_wy_bytes(n) bytes
// of device workspace (the blocks' Gram matrices and triangular factors)
size_t qr64_wy_bytes(int n);
int qr64_form_q(const Launch& L, const z64* V, const z64* tau, int m, int n, z64* Q, long long sQr,
                long long sQc, void* wy);
// one-sided Jacobi on the columns of the M x N column-major A (N even; A is
// overwritten), then the k columns of largest norm copied to out (M x k,
// column-major) in decreasing order of norm: the leading left singular vectors
// of A, each scaled by its singular value. ws: jacobi_ws_bytes(N) bytes;
// a grid barrier that gives up sets *err (code 10).
size_t jacobi_ws_bytes(int N);
int jacobi_top_columns(const Launch& L, z64* A, int M, int N, int k, z64* out, void* ws, int* err);
// R (n x n) from the factored A and beta: dense upper-triangular, row-major
int qr64_extract_r(const Launch& L, const z64* A, const z64* beta, int m, int n, z64* R);

// out[b][s][a] = in[a][s][b] for in of shape [na][d][nb]
int mirror_site64(const Launch& L, const z64* in, z64* out, int na, int d, int nb);
// dst(r, c) = src(r, c) for strided 2-D views (complex)
int copy2d64(const Launch& L, const z64* src, long long sr, long long sc, z64* dst, long long dr,
             long long dc, int rows, int cols);
int fill64(const Launch& L, z64* dst, size_t n, double re, double im);
// dst = the n x n identity (complex, row-major)
int eye64(const Launch& L, z64* dst, int n);
// sum |x|^2 over n entries into *out (device), deterministic two-pass
int norm2_64(const Launch& L, const z64* x, size_t n, double* out, double* scratch);
// x /= sqrt(*nrm2); *lognorm += log(sqrt(*nrm2)); flags nonfinite into *flag
int normalize64(const Launch& L, z64* x, size_t n, const double* nrm2, double* lognorm, int* flag);
// sum_i a[i] * b[i] (no conjugation) into *out (device, complex)
int dotu64(const Launch& L, const z64* a, const z64* b, size_t n, z64* out, double* scratch);
// site densities for local observables of a state whose right transfers are
// identities: rho_partial64 writes site i's block partials of
// rho[s][t] = sum conj(A[a0][s][a]) Y[a0][t][a] (Y = El A, both [Dl][d][Dr],
// d <= 4) to part (rho_part_count(1, d) entries per site), rho_apply64 sums each
// site's partials in a fixed order and writes vals[k][i] = sum_{s,t} O_k[s][t] rho_i[s][t]
size_t rho_part_count(int L, int d);
int rho_partial64(const Launch& L, const z64* A, const z64* Y, int Dl, int d, int Dr, z64* part);
int rho_apply64(const Launch& L, const z64* part, int nsites, int d, const z64* ops, int nops, z64* vals);
// E /= ||E||_F, *logacc += log ||E||_F (overlap transfer rescaling)
int rescale64(const Launch& L, z64* E, size_t n, double* logacc, double* scratch);

}  // namespace tevo
