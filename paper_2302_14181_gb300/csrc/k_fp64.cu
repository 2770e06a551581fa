// fp64 kernels: strided batched complex GEMM with deterministic split-K,
// Householder QR (LAPACK reflector convention, deflation of columns with no
// remaining norm), and the reductions of the fit (norm, rescaling, dot).
//
// GB300 executes fp64 at about 2 DFMA per clock per SM, so every kernel here is
// bound by the fp64 pipe, not by memory: the GEMM keeps one 64x64 complex tile
// per CTA in registers and splits K until every SM has work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cmath>
#include <cstdio>

#include "tevo_internal.h"

namespace tevo {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

constexpr int BM = 64, BN = 64, BK = 16, GEMM_THREADS = 256;

struct GemmKArgs {
  GemmDesc g;
  int splitK;
  int kchunk;
  double2* partial;  // [splitK][batch][M][N] when splitK > 1
};

template <bool CA, bool CB>
__global__ void __launch_bounds__(GEMM_THREADS) zgemm_kernel(GemmKArgs p) {
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const GemmDesc& g = p.g;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int bz = blockIdx.z;
  const int b = bz / p.splitK, sk = bz % p.splitK;
  const int kbeg = sk * p.kchunk;
  const int kend = min(g.K, kbeg + p.kchunk);
  const double2* A = reinterpret_cast<const double2*>(g.A) + (long long)b * g.sAb;
  const double2* B = reinterpret_cast<const double2*>(g.B) + (long long)b * g.sBb;
  const bool a_kfast = (g.sAk == 1);
  const bool b_nfast = (g.sBn == 1);
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / GEMM_THREADS; ++r) {
      int idx = tid + r * GEMM_THREADS;
      int mm, kk;
      if (a_kfast) {
        mm = idx / BK;
        kk = idx % BK;
      } else {
        mm = idx % BM;
        kk = idx / BM;
      }
      int gm = m0 + mm, gk = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (gm < g.M && gk < kend) v = A[(long long)gm * g.sAm + (long long)gk * g.sAk];
      As[kk][mm] = CA ? cconj(v) : v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / GEMM_THREADS; ++r) {
      int idx = tid + r * GEMM_THREADS;
      int nn, kk;
      if (b_nfast) {
        nn = idx % BN;
        kk = idx / BN;
      } else {
        nn = idx / BK;
        kk = idx % BK;
      }
      int gn = n0 + nn, gk = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (gn < g.N && gk < kend) v = B[(long long)gk * g.sBk + (long long)gn * g.sBn];
      Bs[kk][nn] = CB ? cconj(v) : v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (p.splitK > 1) {
    double2* P = p.partial + ((long long)sk * g.batch + b) * (long long)g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm < g.M && gn < g.N) P[(long long)gm * g.N + gn] = acc[i][j];
      }
    return;
  }
  double2* C = reinterpret_cast<double2*>(g.C) + (long long)b * g.sCb;
  const double2 alpha = make_double2(g.alpha_re, g.alpha_im);
  const double2 beta = make_double2(g.beta_re, g.beta_im);
  const bool use_beta = (g.beta_re != 0.0 || g.beta_im != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < g.M && gn < g.N) {
        long long off = (long long)gm * g.sCm + (long long)gn * g.sCn;
        double2 v = cmul(alpha, acc[i][j]);
        if (use_beta) v = cfma(beta, C[off], v);
        C[off] = v;
      }
    }
}

// sum the split-K partials in split order (deterministic) and write C
__global__ void zgemm_reduce_kernel(GemmDesc g, int splitK, const double2* partial) {
  const long long MN = (long long)g.M * g.N;
  const long long total = MN * g.batch;
  const double2 alpha = make_double2(g.alpha_re, g.alpha_im);
  const double2 beta = make_double2(g.beta_re, g.beta_im);
  const bool use_beta = (g.beta_re != 0.0 || g.beta_im != 0.0);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long b = idx / MN, r = idx % MN;
    int m = int(r / g.N), n = int(r % g.N);
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < splitK; ++k) {
      double2 v = partial[((long long)k * g.batch + b) * MN + r];
      s.x += v.x;
      s.y += v.y;
    }
    double2* C = reinterpret_cast<double2*>(g.C) + b * g.sCb;
    long long off = (long long)m * g.sCm + (long long)n * g.sCn;
    double2 v = cmul(alpha, s);
    if (use_beta) v = cfma(beta, C[off], v);
    C[off] = v;
  }
}

void choose_split(const GemmDesc& g, int num_sms, int& splitK, int& kchunk) {
  long long tiles = (long long)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * g.batch;
  splitK = 1;
  long long target = 2LL * num_sms;
  if (tiles < target && g.K > 4 * BK) {
    long long want = (target + tiles - 1) / tiles;
    long long maxs = g.K / (4 * BK);
    splitK = int(want < maxs ? want : maxs);
    if (splitK < 1) splitK = 1;
  }
  kchunk = (g.K + splitK - 1) / splitK;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  splitK = (g.K + kchunk - 1) / kchunk;
  if (splitK < 1) splitK = 1;
}

}  // namespace

size_t zgemm64_workspace(const GemmDesc& g, int num_sms) {
  int splitK, kchunk;
  choose_split(g, num_sms, splitK, kchunk);
  if (splitK <= 1) return 0;
  return sizeof(double2) * (size_t)splitK * g.batch * (size_t)g.M * g.N;
}

int zgemm64(const Launch& L, const GemmDesc& g, void* workspace, size_t ws_bytes) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return 0;
  if (g.K <= 0) return TEVO_EINVAL;
  int splitK, kchunk;
  choose_split(g, L.num_sms, splitK, kchunk);
  size_t need = splitK > 1 ? sizeof(double2) * (size_t)splitK * g.batch * (size_t)g.M * g.N : 0;
  if (need > ws_bytes) {
    splitK = 1;
    kchunk = ((g.K + BK - 1) / BK) * BK;
  }
  if ((long long)g.batch * splitK > 65535 || (g.M + BM - 1) / BM > 65535) return TEVO_ESHAPE;
  GemmKArgs p{g, splitK, kchunk, reinterpret_cast<double2*>(workspace)};
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch * splitK);
  const double flops = 8.0 * g.M * (double)g.N * g.K * g.batch;
  const double bytes = 16.0 * ((double)g.M * g.K * (g.sAb ? g.batch : 1) + (double)g.K * g.N * (g.sBb ? g.batch : 1) +
                               (double)g.M * g.N * g.batch);
  int pr = L.prof ? L.prof->begin(L.stream, TEVO_PROF_GEMM64, flops, bytes) : -1;
  if (g.conjA && g.conjB)
    zgemm_kernel<true, true><<<grid, GEMM_THREADS, 0, L.stream>>>(p);
  else if (g.conjA)
    zgemm_kernel<true, false><<<grid, GEMM_THREADS, 0, L.stream>>>(p);
  else if (g.conjB)
    zgemm_kernel<false, true><<<grid, GEMM_THREADS, 0, L.stream>>>(p);
  else
    zgemm_kernel<false, false><<<grid, GEMM_THREADS, 0, L.stream>>>(p);
  ++*L.launches;
  if (splitK > 1) {
    long long total = (long long)g.M * g.N * g.batch;
    int blocks = int(std::min<long long>((total + 255) / 256, 8LL * L.num_sms));
    zgemm_reduce_kernel<<<blocks, 256, 0, L.stream>>>(g, splitK, p.partial);
    ++*L.launches;
  }
  if (L.prof) L.prof->end(L.stream, pr);
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

// ---------------------------------------------------------------------------
// G2 with the MPO's zero entries skipped
// ---------------------------------------------------------------------------
namespace {

// T_p[r][b] = sum over the nonzeros (r, k) of W: W[r][k] * X_p[k][b].
// One CTA per (p, block of BW columns b): X_p[:, block] is staged in shared
// memory; a warp walks the nonzeros of one row r for 32 consecutive b.
// The nonzeros of a row are visited in increasing k, the order in which the
// dense kernel accumulates them, and skipped entries are exact zeros, so the
// result equals the dense contraction bit for bit.
__global__ void __launch_bounds__(256) zsparse_g2_kernel(const double2* __restrict__ X, double2* __restrict__ T,
                                                         const int* __restrict__ row_ptr,
                                                         const int* __restrict__ col_idx,
                                                         const double2* __restrict__ vals, int R, int K, int Db,
                                                         int BW) {
  extern __shared__ double2 xs[];  // [K][BW]
  const int p = blockIdx.y;
  const int b0 = blockIdx.x * BW;
  const int bw = min(BW, Db - b0);
  const double2* Xp = X + (long long)p * K * Db;
  for (int idx = threadIdx.x; idx < K * BW; idx += blockDim.x) {
    const int k = idx / BW, bb = idx % BW;
    xs[idx] = (bb < bw) ? Xp[(long long)k * Db + b0 + bb] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  double2* Tp = T + (long long)p * R * Db;
  const int lanes = min(BW, 32);
  const int per_block = blockDim.x / lanes;  // rows processed at once
  const int bb = threadIdx.x % lanes, rsub = threadIdx.x / lanes;
  for (int r = rsub; r < R; r += per_block) {
    for (int bc = bb; bc < bw; bc += lanes) {
      double2 acc = make_double2(0.0, 0.0);
      for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) acc = cfma(vals[e], xs[col_idx[e] * BW + bc], acc);
      Tp[(long long)r * Db + b0 + bc] = acc;
    }
  }
}

}  // namespace

int zsparse_g2(const Launch& L, const z64* X, z64* T, const int* row_ptr, const int* col_idx, const z64* vals,
               int R, int K, int Db, int batch) {
  int BW = 32;
  while (BW > 8 && (size_t)K * BW * sizeof(double2) > 200 * 1024) BW /= 2;
  const size_t smem = (size_t)K * BW * sizeof(double2);
  if (smem > 220 * 1024) return TEVO_EUNSUPPORTED;
  static std::atomic<unsigned long long> attr{0};
  if (smem_attr_once(zsparse_g2_kernel, 220 * 1024, attr)) return TEVO_ECUDA;
  if (batch > 65535) return TEVO_ESHAPE;
  dim3 grid((Db + BW - 1) / BW, batch);
  zsparse_g2_kernel<<<grid, 256, smem, L.stream>>>(reinterpret_cast<const double2*>(X), reinterpret_cast<double2*>(T),
                                                    row_ptr, col_idx, reinterpret_cast<const double2*>(vals), R, K,
                                                    Db, BW);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

// ---------------------------------------------------------------------------
// Householder QR
// ---------------------------------------------------------------------------
namespace {

constexpr int QR_THREADS = 128;
// upper bound on the CTAs of the cooperative factorisation (compile-time choice)
#ifndef QR_COOP_MAX_CTAS
#define QR_COOP_MAX_CTAS 1024
#endif
constexpr double DEFLATE = 2.2737367544323206e-13;  // 2^-42
constexpr int JAC_MAX_SWEEPS = 40;
constexpr double JAC_TOL = 1e-15;

// Block reductions. Lane 0 of each warp ends with the warp's sum; at offset o
// only lanes below o feed a lane that a later offset reads, so the others skip
// the add (lane 0's sum is that of the full tree). Thread 0 adds the warps'
// sums in a fixed order and shares the total through shared memory: the
// scalar fp64 work runs once per block, not once per thread. Blocks of at most
// 512 threads (red[16] and red[48] hold the shared totals).
__device__ __forceinline__ double warp_sum0(double v) {
  const int lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane < o) v += u;
  }
  return v;
}

__device__ __forceinline__ double2 warp_csum0(double2 v) {
  const int lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) {
    const double ux = __shfl_down_sync(0xffffffffu, v.x, o);
    const double uy = __shfl_down_sync(0xffffffffu, v.y, o);
    if (lane < o) {
      v.x += ux;
      v.y += uy;
    }
  }
  return v;
}

// the warps' sums of v into red[0..nw) (thread 0 reads them after the barrier)
__device__ __forceinline__ void block_partials(double v, double* red) {
  v = warp_sum0(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
}

__device__ __forceinline__ double total_of(const double* red) {
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) s += red[w];  // fixed order
  return s;
}

__device__ double block_sum(double v, double* red) {
  block_partials(v, red);
  if (threadIdx.x == 0) red[16] = total_of(red);
  __syncthreads();
  return red[16];
}

// a * (the block's sum of v), for every thread; a = 1 gives the plain sum
// (both parts summed in block_sum's order, one round of barriers)
__device__ double2 block_csum_times(double2 v, double2 a, double* red, bool scale) {
  v = warp_csum0(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = v.x;
    red[32 + (threadIdx.x >> 5)] = v.y;
  }
  __syncthreads();
  if (threadIdx.x < 2) {  // lane 0 adds the real parts, lane 1 the imaginary ones
    const double p = total_of(red + 32 * threadIdx.x);
    const double q = __shfl_sync(0x3u, p, 1);
    if (threadIdx.x == 0) {
      double2 s = make_double2(p, q);
      if (scale) s = cmul(a, s);
      red[16] = s.x;
      red[48] = s.y;
    }
  }
  __syncthreads();
  return make_double2(red[16], red[48]);
}

__device__ double2 block_csum(double2 v, double* red) {
  return block_csum_times(v, make_double2(1.0, 0.0), red, false);
}

// the same sums, with every thread adding the warps' totals itself (no third
// barrier): the better trade where many blocks share a multiprocessor
__device__ double2 block_csum_every(double2 v, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[wid] = v.x;
    red[32 + wid] = v.y;
  }
  __syncthreads();
  return make_double2(total_of(red), total_of(red + 32));
}

// sum |A|^2 of the m x n matrix (partial sums per block, fixed grid)
__global__ void frob_partial_kernel(const double2* A, long long n, double* part) {
  __shared__ double red[64];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 v = A[i];
    s = fma(v.x, v.x, s);
    s = fma(v.y, v.y, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_partials_kernel(const double* part, int np, double* out) {
  __shared__ double red[64];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

constexpr int FROB_BLOCKS = 256;

// One column step k. Every CTA recomputes the reflector of column k from the
// (already updated) column, then applies H_k^H to one trailing column j.
// CTA 0 with j == k+1 (or the only CTA when k == n-1) records v, tau, beta.
__global__ void qr_step_kernel(double2* A, int m, int n, int k, double2* V, double2* tau,
                               double2* beta, const double* frob2) {
  extern __shared__ double2 v[];  // m - k entries
  __shared__ double red[64];
  const int len = m - k;
  const double2* x = A + (long long)k * m + k;
  double s = 0.0;
  for (int r = threadIdx.x; r < len; r += blockDim.x) {
    double2 a = x[r];
    v[r] = a;
    s = fma(a.x, a.x, s);
    s = fma(a.y, a.y, s);
  }
  const double nrm2 = block_sum(s, red);
  const double nrm = sqrt(nrm2);
  const double tol = DEFLATE * sqrt(*frob2);
  const double2 alpha = v[0];
  const bool deflate = (nrm <= tol) || (nrm == 0.0);
  double2 t = make_double2(0.0, 0.0);
  double b = 0.0;
  if (!deflate) {
    b = alpha.x >= 0.0 ? -nrm : nrm;
    t = make_double2((b - alpha.x) / b, -alpha.y / b);
    // v = x / (alpha - beta), v[0] = 1
    double2 den = make_double2(alpha.x - b, alpha.y);
    double dd = den.x * den.x + den.y * den.y;
    double2 inv = make_double2(den.x / dd, -den.y / dd);
    __syncthreads();
    for (int r = threadIdx.x; r < len; r += blockDim.x) v[r] = (r == 0) ? make_double2(1.0, 0.0) : cmul(v[r], inv);
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      tau[k] = t;
      beta[k] = deflate ? alpha : make_double2(b, 0.0);
    }
    double2* Vk = V + (long long)k * m;
    for (int r = threadIdx.x; r < m; r += blockDim.x)
      Vk[r] = (r < k) ? make_double2(0.0, 0.0) : (deflate ? make_double2(r == k ? 1.0 : 0.0, 0.0) : v[r - k]);
  }
  if (deflate) return;
  const int j = k + 1 + blockIdx.x;
  if (j >= n) return;
  double2* col = A + (long long)j * m + k;
  // w = v^H col
  double2 w = make_double2(0.0, 0.0);
  for (int r = threadIdx.x; r < len; r += blockDim.x) w = cfma(cconj(v[r]), col[r], w);
  // col -= conj(t) v w
  const double2 f = block_csum_times(w, cconj(t), red, true);
  for (int r = threadIdx.x; r < len; r += blockDim.x) {
    double2 c = col[r];
    double2 d = cmul(v[r], f);
    col[r] = make_double2(c.x - d.x, c.y - d.y);
  }
}

// ---------------------------------------------------------------------------
// Explicit thin Q from the compact WY form of blocks of reflectors
// (Schreiber - Van Loan): H_j0 H_j0+1 ... H_j1-1 = I - V_b T_b V_b^H with T_b
// upper triangular, T[i][i] = tau_i and T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i],
// G = V_b^H V_b. Column c of Q is the product of the blocks b = c / WY_NB ... 0
// applied, last block first, to e_c, so that each block costs one reduction
// round (WY_NB dot products together) instead of WY_NB dependent ones.
// ---------------------------------------------------------------------------
constexpr int WY_NB = 16;
constexpr int WY_GRAM_SPLIT = 8;  // CTAs sharing the dot products of one block

// G[b][i][j] = v_{j0+i}^H v_{j0+j} for i < j within block b (row >= j0 + j,
// where v_{j0+j} starts); CTA (b, s) takes the pairs p = s, s + SPLIT, ...
// one warp per pair
__global__ void qr_wy_gram_kernel(const double2* V, int m, int n, double2* G) {
  const int b = blockIdx.x, j0 = b * WY_NB, nbk = min(WY_NB, n - j0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int npair = nbk * (nbk - 1) / 2;
  for (int p = blockIdx.y + WY_GRAM_SPLIT * warp; p < npair; p += WY_GRAM_SPLIT * nw) {
    // p -> (i, j), i < j, row-major over the strict upper triangle
    int i = 0, rem = p;
    while (rem >= nbk - 1 - i) {
      rem -= nbk - 1 - i;
      ++i;
    }
    const int j = i + 1 + rem;
    const double2* vi = V + (long long)(j0 + i) * m;
    const double2* vj = V + (long long)(j0 + j) * m;
    double2 sum = make_double2(0.0, 0.0);
    for (int r = j0 + j + lane; r < m; r += 32) sum = cfma(cconj(vi[r]), vj[r], sum);
    sum = warp_csum0(sum);
    if (lane == 0) G[((size_t)b * WY_NB + i) * WY_NB + j] = sum;
  }
}

// T_b from G_b and tau (one warp per block): G_b and the block's tau are staged
// in shared memory, then column i of T is formed after columns 0..i-1; lane
// r < i forms T[r][i]
__global__ void qr_wy_t_kernel(const double2* tau, int n, const double2* G, double2* Tf) {
  __shared__ double2 T[WY_NB][WY_NB];
  __shared__ double2 Gs[WY_NB][WY_NB];
  __shared__ double2 ts[WY_NB];
  const int b = blockIdx.x, j0 = b * WY_NB, nbk = min(WY_NB, n - j0);
  const int lane = threadIdx.x;
  const double2* Gb = G + (size_t)b * WY_NB * WY_NB;
  for (int e = lane; e < WY_NB * WY_NB; e += 32) {
    const int r = e / WY_NB, c = e % WY_NB;
    Gs[r][c] = r < c && c < nbk ? Gb[e] : make_double2(0.0, 0.0);  // only the strict upper part is formed
  }
  if (lane < nbk) ts[lane] = tau[j0 + lane];
  __syncwarp();
  for (int i = 0; i < nbk; ++i) {
    const double2 ti = ts[i];
    double2 t = make_double2(0.0, 0.0);
    if (lane < i) {
      // sum_{k = lane}^{i-1} T[lane][k] G[k][i] (T upper triangular)
      for (int k = lane; k < i; ++k) t = cfma(T[lane][k], Gs[k][i], t);
      t = cmul(make_double2(-ti.x, -ti.y), t);
    } else if (lane == i) {
      t = ti;
    }
    __syncwarp();
    if (lane < WY_NB) T[lane][i] = lane <= i ? t : make_double2(0.0, 0.0);
    __syncwarp();
  }
  for (int e = lane; e < WY_NB * WY_NB; e += 32) {
    const int r = e / WY_NB, c = e % WY_NB;
    Tf[(size_t)b * WY_NB * WY_NB + e] = (r < nbk && c < nbk) ? T[r][c] : make_double2(0.0, 0.0);
  }
}

// column c of Q (one CTA per column; the first `heavy` blocks take the most
// expensive columns and the rest the cheapest ones, so that blocks sharing a
// multiprocessor pair a long column with a short one): q = e_c, then for b = c / WY_NB down to 0:
// w = V_b^H q (warp i takes the dot products of reflectors i, i + nw, ...),
// w' = T_b w, q -= V_b w'. Within block c / WY_NB only the reflectors up to c
// act on e_c.
__global__ void qr_wy_form_kernel(const double2* V, int m, int n, const double2* Tf, double2* Q, long long sQr,
                                  long long sQc, int heavy) {
  extern __shared__ double2 q[];
  __shared__ double2 w[WY_NB], wp[WY_NB];
  const int c = (int)blockIdx.x < heavy ? n - 1 - (int)blockIdx.x : (int)blockIdx.x - heavy;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = threadIdx.x; r < m; r += blockDim.x) q[r] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int b = c / WY_NB; b >= 0; --b) {
    const int j0 = b * WY_NB;
    const int nb = b == c / WY_NB ? c - j0 + 1 : min(WY_NB, n - j0);
    for (int i = warp; i < nb; i += nw) {
      const double2* vi = V + (long long)(j0 + i) * m;
      double2 sum = make_double2(0.0, 0.0);
      for (int r = j0 + i + lane; r < m; r += 32) sum = cfma(cconj(vi[r]), q[r], sum);
      sum = warp_csum0(sum);
      if (lane == 0) w[i] = sum;
    }
    __syncthreads();
    if (threadIdx.x < nb) {
      const double2* Tb = Tf + (size_t)b * WY_NB * WY_NB + (size_t)threadIdx.x * WY_NB;
      double2 t = make_double2(0.0, 0.0);
      for (int k = threadIdx.x; k < nb; ++k) t = cfma(Tb[k], w[k], t);
      wp[threadIdx.x] = t;
    }
    __syncthreads();
    for (int r = j0 + threadIdx.x; r < m; r += blockDim.x) {
      double2 acc = q[r];
      const int imax = min(nb, r - j0 + 1);  // v_{j0+i} is zero above row j0 + i
      for (int i = 0; i < imax; ++i) {
        const double2 d = cmul(V[(long long)(j0 + i) * m + r], wp[i]);
        acc.x -= d.x;
        acc.y -= d.y;
      }
      q[r] = acc;
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < m; r += blockDim.x) Q[(long long)r * sQr + (long long)c * sQc] = q[r];
}

// Householder scalars of a column (shared by every thread of the block)
struct Refl {
  double2 inv;   // 1 / (alpha - beta), the scale of the column below its first row
  double2 tau;
  double2 beta;
  int deflate;
};

// The block's total of the per-thread squares s and the reflector of a column
// whose first entry is alpha (read in thread 0 only). Lanes 0..3 of warp 0 form
// the scalars (deflation as in qr_step_kernel): each adds the same total and
// takes the same square root, then each takes one of the four independent
// quotients; thread 0 shares the result with the block.
__device__ Refl block_reflector(double s, double2 alpha, double tol, double* red, Refl* sr) {
  block_partials(s, red);
  if (threadIdx.x < 4) {
    const unsigned lanes = 0xfu;
    const int l = threadIdx.x;
    const double ax = __shfl_sync(lanes, alpha.x, 0), ay = __shfl_sync(lanes, alpha.y, 0);
    const double nrm = sqrt(total_of(red));
    const double b = ax >= 0.0 ? -nrm : nrm;
    const double2 den = make_double2(ax - b, ay);
    const double dd = den.x * den.x + den.y * den.y;
    // inv = (den.x / dd, -den.y / dd), tau = ((b - ax) / b, -ay / b); unused
    // (and possibly not finite) when the column deflates
    const double num = l == 0 ? den.x : l == 1 ? -den.y : l == 2 ? b - ax : -ay;
    const double q = num / (l < 2 ? dd : b);
    const double q1 = __shfl_sync(lanes, q, 1), q2 = __shfl_sync(lanes, q, 2), q3 = __shfl_sync(lanes, q, 3);
    if (l == 0) {
      Refl R;
      R.deflate = (nrm <= tol) || (nrm == 0.0);
      if (R.deflate) {
        R.inv = make_double2(0.0, 0.0);
        R.tau = make_double2(0.0, 0.0);
        R.beta = make_double2(ax, ay);
      } else {
        R.inv = make_double2(q, q1);
        R.tau = make_double2(q2, q3);
        R.beta = make_double2(b, 0.0);
      }
      *sr = R;
    }
  }
  __syncthreads();
  return *sr;
}

// reflector of the column x[k..m) (in shared memory) into vout[k..m) and the
// global copy vg[k..m)
__device__ Refl make_reflector(const double2* x, double2* vout, double2* vg, int k, int m, double tol,
                               double* red, Refl* sr) {
  double s = 0.0;
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
    double2 a = x[r];
    s = fma(a.x, a.x, s);
    s = fma(a.y, a.y, s);
  }
  const Refl R = block_reflector(s, x[k], tol, red, sr);
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
    const double2 e = R.deflate ? make_double2(r == k ? 1.0 : 0.0, 0.0)
                                : ((r == k) ? make_double2(1.0, 0.0) : cmul(x[r], R.inv));
    vout[r] = e;
    vg[r] = e;
  }
  return R;
}

// col[k..m) -= conj(tau) v (v^H col[k..m))
__device__ void apply_reflector(double2* col, const double2* v, double2 tau, int k, int m, double* red) {
  if (tau.x == 0.0 && tau.y == 0.0) return;  // uniform across the block
  double2 w = make_double2(0.0, 0.0);
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) w = cfma(cconj(v[r]), col[r], w);
  const double2 f = block_csum_times(w, cconj(tau), red, true);
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
    double2 d = cmul(v[r], f);
    col[r] = make_double2(col[r].x - d.x, col[r].y - d.y);
  }
  __syncthreads();
}

// the look-ahead step of the owner of column k1 = k + 1: apply reflector k to
// that column and form reflector k1 from the result (into vout and its global
// copy vg), with two block reductions. Every sum runs over the rows in the
// order apply_reflector and make_reflector use, so the result is bitwise that
// of those two calls. Thread 0 updates row k and holds row k1 (alpha).
__device__ Refl apply_then_reflect(double2* col, const double2* v, double2 t, int k, int m, double tol,
                                   double2* vout, double2* vg, double* red, Refl* sr) {
  const int k1 = k + 1;
  const bool act = !(t.x == 0.0 && t.y == 0.0);  // uniform across the block
  double2 f = make_double2(0.0, 0.0);
  if (act) {
    double2 w = make_double2(0.0, 0.0);
    for (int r = k + threadIdx.x; r < m; r += blockDim.x) w = cfma(cconj(v[r]), col[r], w);
    f = block_csum_times(w, cconj(t), red, true);
  }
  if (act && threadIdx.x == 0) {  // row k: the R entry of the column
    const double2 d = cmul(v[k], f);
    col[k] = make_double2(col[k].x - d.x, col[k].y - d.y);
  }
  double s = 0.0;
  double2 alpha = make_double2(0.0, 0.0);
  for (int r = k1 + threadIdx.x; r < m; r += blockDim.x) {
    double2 x = col[r];
    if (act) {
      const double2 d = cmul(v[r], f);
      x = make_double2(x.x - d.x, x.y - d.y);
      col[r] = x;
    }
    s = fma(x.x, x.x, s);
    s = fma(x.y, x.y, s);
    if (r == k1) alpha = x;
  }
  const Refl R = block_reflector(s, alpha, tol, red, sr);
  // each thread scales the rows it updated above
  for (int r = k1 + threadIdx.x; r < m; r += blockDim.x) {
    const double2 e = R.deflate ? make_double2(r == k1 ? 1.0 : 0.0, 0.0)
                                : ((r == k1) ? make_double2(1.0, 0.0) : cmul(col[r], R.inv));
    vout[r] = e;
    vg[r] = e;
  }
  return R;
}

// Cooperative Householder factorisation, one launch for all columns. CTA c owns
// columns j = c, c + G, c + 2G, ... (G = grid size), kept in shared memory. At
// step k the owner of column k publishes reflector k (V[k.., k], tau_k in
// V[k - 1, k], tau[k], beta[k]), every other CTA acquires it and applies H_k^H
// to its own columns > k. V starts filled with a value no entry can take, so a
// consumer polls the entries it reads until they are written (no flag and
// second round trip); reflector 0 alone, which has no row above it, is
// published by a release flag. The owner of column k + 1 updates that column first
// and publishes reflector k + 1 before updating its other columns, so the chain
// of dependent work per step is one column update plus one norm; the rows of
// V above the diagonal and the R part of the column, which only later kernels
// read, are written after the release. All CTAs are co-resident (cooperative
// launch); every wait is bounded (err, code 8) and, after a timeout, all CTAs
// leave.
constexpr unsigned long long QR_WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long qr_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// V is filled with this byte pattern (0x7F in every byte, about 1.38e306 as a
// double) before the factorisation. No entry of a reflector (|v_r| <= 1, the
// scale of a column by 1 / (alpha - beta) with |alpha - beta| >= |x|), of a tau
// (|tau| <= 2) or of the zeros above can equal it, so an entry of V that no
// longer holds it in both halves has its final value: a consumer polls the rows
// it reads instead of a flag and then the rows.
constexpr unsigned long long QR_V_UNSET = 0x7F7F7F7F7F7F7F7Full;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// the entry at p once both of its halves are written; false after the time
// limit (err set to code)
__device__ bool poll_entry(const double2* p, double2& out, int* err, int code) {
  unsigned long long re = ld_relaxed_u64(&p->x), im = ld_relaxed_u64(&p->y);
  if (re == QR_V_UNSET || im == QR_V_UNSET) {
    const unsigned long long t0 = qr_gtimer();
    while (re == QR_V_UNSET || im == QR_V_UNSET) {
      if (qr_gtimer() - t0 > QR_WAIT_NS) {
        atomicExch(err, code);
        return false;
      }
      if (re == QR_V_UNSET) re = ld_relaxed_u64(&p->x);
      if (im == QR_V_UNSET) im = ld_relaxed_u64(&p->y);
    }
  }
  out = make_double2(__longlong_as_double((long long)re), __longlong_as_double((long long)im));
  return true;
}

__global__ void __launch_bounds__(256) qr_coop_kernel(double2* A, int m, int n, double2* V, double2* tau,
                                                      double2* beta, const double* frob2, int* flags, int epoch,
                                                      int* err) {
  extern __shared__ double2 sm[];
  __shared__ double red[64];
  __shared__ double2 s_tau[2];
  __shared__ Refl s_refl;
  __shared__ int s_abort;
  const int G = gridDim.x, c = blockIdx.x;
  const int ncols = (n - c + G - 1) / G;  // columns owned
  double2* cols = sm;                      // [ncols][m]
  double2* vb[2] = {sm + (size_t)ncols * m, sm + (size_t)(ncols + 1) * m};
  const double tol = DEFLATE * sqrt(*frob2);
  for (int jj = 0; jj < ncols; ++jj) {
    const int j = c + jj * G;
    for (int r = threadIdx.x; r < m; r += blockDim.x) cols[(size_t)jj * m + r] = A[(long long)j * m + r];
  }
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  // release reflector k, whose rows k.. of V are already stored by the threads
  // that formed them (called by the owner of column k with s_refl holding its
  // scalars)
  auto release = [&](int k) {
    if (threadIdx.x == 0) {
      s_tau[k & 1] = s_refl.tau;
      tau[k] = s_refl.tau;
      beta[k] = s_refl.beta;
      // tau_k also rides in row k - 1 of V's column k (above the reflector, a
      // row no reader of V uses otherwise), so a consumer fetches it together
      // with the reflector's rows instead of in a dependent load of its own
      if (k > 0) V[(long long)k * m + k - 1] = s_refl.tau;
    }
    // the block barrier orders every thread's stores of V before thread 0's
    // release store, which is cumulative over them (reflector 0 only: the
    // consumers of the others poll V itself), and publishes s_tau to the block
    __syncthreads();
    if (threadIdx.x == 0 && k == 0) st_release(flags + k, epoch);
    // rows above k - 1: zeros of V, and the R part of column k for qr64_extract_r
    const double2* col = cols + (size_t)(k / G) * m;
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
      if (r + 1 < k) V[(long long)k * m + r] = make_double2(0.0, 0.0);
      A[(long long)k * m + r] = col[r];
    }
  };
  // the owner of column 0 starts the chain
  if (c == 0) {
    make_reflector(cols, vb[0], V, 0, m, tol, red, &s_refl);
    release(0);
  }
  for (int k = 0; k < n; ++k) {
    const int owner = k % G;
    double2* v = vb[k & 1];
    if (owner != c && k > 0) {
      // reflector k: each thread polls the rows of V_k it reads first (its own
      // rows of the dot products below), and the last thread tau_k in row
      // k - 1; other threads read them only after a reduction's barrier
      const double2* Vk = V + (long long)k * m;
      bool ok = true;
      for (int r = k + threadIdx.x; r < m && ok; r += blockDim.x) ok = poll_entry(Vk + r, v[r], err, 8);
      if (ok && threadIdx.x == blockDim.x - 1) {
        double2 t;
        ok = poll_entry(Vk + k - 1, t, err, 8);
        s_tau[k & 1] = t;
      }
      if (!ok) s_abort = 1;
      __syncthreads();
      if (s_abort) return;
    } else if (owner != c) {
      // reflector 0 (no row above it for tau): acquire its flag
      if (threadIdx.x == 0) {
        if (ld_acquire(flags + k) != epoch) {
          const unsigned long long t0 = qr_gtimer();
          while (ld_acquire(flags + k) != epoch) {
            if (qr_gtimer() - t0 > QR_WAIT_NS) {
              atomicExch(err, 8);
              s_abort = 1;
              break;
            }
          }
        }
      }
      __syncthreads();
      if (s_abort) return;
      const double2* Vk = V + (long long)k * m;
      for (int r = k + threadIdx.x; r < m; r += blockDim.x) v[r] = __ldcg(Vk + r);  // L2, never a stale L1 line
      if (threadIdx.x == blockDim.x - 1) s_tau[k & 1] = __ldcg(tau);
      __syncthreads();
    }
    const double2 t = s_tau[k & 1];
    // look-ahead: column k + 1 first, then publish reflector k + 1
    const int k1 = k + 1;
    if (k1 < n && (k1 % G) == c) {
      double2* col = cols + (size_t)(k1 / G) * m;
      apply_then_reflect(col, v, t, k, m, tol, vb[k1 & 1], V + (long long)k1 * m, red, &s_refl);
      release(k1);
    }
    for (int jj = 0; jj < ncols; ++jj) {
      const int j = c + jj * G;
      if (j <= k || j == k1) continue;
      apply_reflector(cols + (size_t)jj * m, v, t, k, m, red);
    }
  }
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of an M x N complex matrix
// (column-major, ld = M, N even): rotations of column pairs until every pair
// is orthogonal to |x^H y| <= tol sqrt(|x|^2 |y|^2); the columns then are the
// left singular vectors scaled by the singular values. One cooperative launch:
// each round takes N/2 disjoint pairs (the circle ordering: position 0 fixed,
// the others rotating, so every pair meets once per sweep of N - 1 rounds),
// CTA c the pairs c, c + G, ...; the rounds are separated by a grid barrier on
// a global counter (bounded wait, err code 10). A sweep without any rotation
// ends the loop (a vote in votes[sweep], zeroed before the launch).
//
// For columns x, y with a = |x|^2, b = |y|^2, c = x^H y = |c| w:
// zeta = (b - a) / (2|c|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// cs = 1 / sqrt(1 + t^2), sn = cs t, and
// x' = cs x - sn conj(w) y,  y' = sn w x + cs y   (x'^H y' = 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int jac_pos(int j, int r, int N) {
  return j == 0 ? 0 : 1 + (j - 1 + r) % (N - 1);
}

__device__ bool jac_barrier(unsigned int* bar, unsigned int target, int* err) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    if (ld_acquire(reinterpret_cast<const int*>(bar)) < (int)target) {
      const unsigned long long t0 = qr_gtimer();
      while (ld_acquire(reinterpret_cast<const int*>(bar)) < (int)target) {
        if (qr_gtimer() - t0 > QR_WAIT_NS) {
          atomicExch(err, 10);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(256) jacobi_cols_kernel(double2* A, int M, int N, int maxsweeps, double tol,
                                                          const double* frob2, unsigned int* bar, int* votes,
                                                          int* err) {
  __shared__ double red[4][8];
  __shared__ double sc[4];
  const int G = gridDim.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // columns below 2^-50 of the matrix's Frobenius norm are rounding residue
  // (rank deficiency): they are not rotated
  const double small = *frob2 * 7.888609052210118e-31;  // 2^-100
  unsigned int nbar = 0;
  for (int sweep = 0; sweep < maxsweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int pi = blockIdx.x; pi < N / 2; pi += G) {
        const int u = jac_pos(pi, r, N), v = jac_pos(N - 1 - pi, r, N);
        const int p = min(u, v), q = max(u, v);
        double2* x = A + (long long)p * M;
        double2* y = A + (long long)q * M;
        double sa = 0.0, sb = 0.0, cr = 0.0, ci = 0.0;
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
          const double2 xi = __ldcg(x + i), yi = __ldcg(y + i);
          sa = fma(xi.x, xi.x, fma(xi.y, xi.y, sa));
          sb = fma(yi.x, yi.x, fma(yi.y, yi.y, sb));
          cr = fma(xi.x, yi.x, fma(xi.y, yi.y, cr));   // Re conj(x) y
          ci = fma(xi.x, yi.y, fma(-xi.y, yi.x, ci));  // Im conj(x) y
        }
        for (int o = 16; o > 0; o >>= 1) {
          sa += __shfl_xor_sync(0xffffffffu, sa, o);
          sb += __shfl_xor_sync(0xffffffffu, sb, o);
          cr += __shfl_xor_sync(0xffffffffu, cr, o);
          ci += __shfl_xor_sync(0xffffffffu, ci, o);
        }
        if (lane == 0) {
          red[0][wid] = sa;
          red[1][wid] = sb;
          red[2][wid] = cr;
          red[3][wid] = ci;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
          double t = 0.0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];  // fixed order
          sc[threadIdx.x] = t;
        }
        __syncthreads();
        const double a = sc[0], b = sc[1], c_re = sc[2], c_im = sc[3];
        const double g = sqrt(c_re * c_re + c_im * c_im);
        if (a > small && b > small && g > tol * sqrt(a) * sqrt(b)) {
          rotated = 1;
          const double zeta = (b - a) / (2.0 * g);
          const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                              : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          const double wr = c_re / g, wi = c_im / g;  // w = c / |c|
          for (int i = threadIdx.x; i < M; i += blockDim.x) {
            const double2 xi = __ldcg(x + i), yi = __ldcg(y + i);
            // conj(w) y = (wr yr + wi yi, wr yi - wi yr);  w x = (wr xr - wi xi, wr xi + wi xr)
            const double2 cy = make_double2(wr * yi.x + wi * yi.y, wr * yi.y - wi * yi.x);
            const double2 wx = make_double2(wr * xi.x - wi * xi.y, wr * xi.y + wi * xi.x);
            __stcg(x + i, make_double2(cs * xi.x - sn * cy.x, cs * xi.y - sn * cy.y));
            __stcg(y + i, make_double2(sn * wx.x + cs * yi.x, sn * wx.y + cs * yi.y));
          }
        }
        __syncthreads();
      }
      if (!jac_barrier(bar, (++nbar) * (unsigned int)G, err)) return;
    }
    if (threadIdx.x == 0 && rotated) atomicOr(votes + sweep, 1);
    if (!jac_barrier(bar, (++nbar) * (unsigned int)G, err)) return;
    if (ld_acquire(votes + sweep) == 0) return;  // every CTA reads the same settled vote
  }
}

// squared norms of the N columns (a warp per column)
__global__ void col_norms_kernel(const double2* A, int M, int N, double* nrm) {
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < N; c += gridDim.x * (blockDim.x >> 5)) {
    double s = 0.0;
    for (int i = lane; i < M; i += 32) {
      const double2 v = A[(long long)c * M + i];
      s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[c] = s;
  }
}

// column j goes to output column rank(j) when rank(j) < k, rank = the number
// of columns with a larger norm (ties: lower index first): the k columns of
// largest norm in decreasing order
__global__ void gather_top_kernel(const double2* A, int M, int N, const double* nrm, int k, double2* out) {
  const int j = blockIdx.x;
  __shared__ int s_rank;
  if (threadIdx.x == 0) s_rank = 0;
  __syncthreads();
  const double nj = nrm[j];
  int cnt = 0;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const double nc = nrm[c];
    cnt += (nc > nj || (nc == nj && c < j)) ? 1 : 0;
  }
  atomicAdd(&s_rank, cnt);
  __syncthreads();
  const int rk = s_rank;
  if (rk >= k) return;
  for (int i = threadIdx.x; i < M; i += blockDim.x) out[(long long)rk * M + i] = A[(long long)j * M + i];
}

__global__ void qr_extract_r_kernel(const double2* A, const double2* beta, int m, int n, double2* R) {
  long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int r = int(idx / n), c = int(idx % n);
    double2 v = make_double2(0.0, 0.0);
    if (r == c)
      v = beta[r];
    else if (r < c)
      v = A[(long long)c * m + r];
    R[idx] = v;
  }
}

}  // namespace

size_t qr64_scratch_bytes(int m, int n) { return sizeof(double) * (FROB_BLOCKS + 8); }

int qr64_factor(const Launch& L, z64* A_, int m, int n, z64* V_, z64* tau_, z64* beta_, void* scratch) {
  if (m < n || n <= 0) return TEVO_ESHAPE;
  double2* A = reinterpret_cast<double2*>(A_);
  double2* V = reinterpret_cast<double2*>(V_);
  double2* tau = reinterpret_cast<double2*>(tau_);
  double2* beta = reinterpret_cast<double2*>(beta_);
  double* part = reinterpret_cast<double*>(scratch);
  double* frob2 = part + FROB_BLOCKS;
  const double qflops = 8.0 * ((double)m * n * n - (double)n * n * n / 3.0);
  int pr = L.prof ? L.prof->begin(L.stream, TEVO_PROF_QR, qflops, 32.0 * (double)m * n) : -1;
  frob_partial_kernel<<<FROB_BLOCKS, 256, 0, L.stream>>>(A, (long long)m * n, part);
  sum_partials_kernel<<<1, 256, 0, L.stream>>>(part, FROB_BLOCKS, frob2);
  *L.launches += 2;
  const size_t smem = sizeof(double2) * (size_t)m;
  if (smem > 48 * 1024) {
    static std::atomic<unsigned long long> attr_step{0};
    if (smem_attr_once(qr_step_kernel, 200 * 1024, attr_step)) return TEVO_ECUDA;
  }
  for (int k = 0; k < n; ++k) {
    int grid = n - k - 1;
    if (grid < 1) grid = 1;
    qr_step_kernel<<<grid, QR_THREADS, smem, L.stream>>>(A, m, n, k, V, tau, beta, frob2);
    ++*L.launches;
  }
  if (L.prof) L.prof->end(L.stream, pr);
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int qr64_factor_coop(const Launch& L, z64* A_, int m, int n, z64* V_, z64* tau_, z64* beta_, void* scratch,
                     int* flags, int epoch, int* err) {
  if (m < n || n <= 0) return TEVO_ESHAPE;
  double2* A = reinterpret_cast<double2*>(A_);
  double* part = reinterpret_cast<double*>(scratch);
  double* frob2 = part + FROB_BLOCKS;
  const int G = std::min({n, L.num_sms, QR_COOP_MAX_CTAS});
  const int ncols = (n + G - 1) / G;
  const size_t smem = sizeof(double2) * (size_t)(ncols + 2) * m;
  if (smem > 200 * 1024) return TEVO_EUNSUPPORTED;
  static std::atomic<unsigned long long> attr{0};
  if (smem_attr_once(qr_coop_kernel, 200 * 1024, attr)) return TEVO_ECUDA;
  // every CTA must be resident at once: check the occupancy for this size
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_coop_kernel, 256, smem) != cudaSuccess ||
      per_sm * L.num_sms < G)
    return TEVO_EUNSUPPORTED;
  const double qflops = 8.0 * ((double)m * n * n - (double)n * n * n / 3.0);
  int pr = L.prof ? L.prof->begin(L.stream, TEVO_PROF_QR, qflops, 32.0 * (double)m * n) : -1;
  frob_partial_kernel<<<FROB_BLOCKS, 256, 0, L.stream>>>(A, (long long)m * n, part);
  sum_partials_kernel<<<1, 256, 0, L.stream>>>(part, FROB_BLOCKS, frob2);
  *L.launches += 2;
  double2* V = reinterpret_cast<double2*>(V_);
  double2* tau = reinterpret_cast<double2*>(tau_);
  double2* beta = reinterpret_cast<double2*>(beta_);
  // every entry of V starts as QR_V_UNSET (the kernel writes all of them)
  if (cudaMemsetAsync(V, 0x7F, sizeof(double2) * (size_t)m * n, L.stream) != cudaSuccess) return TEVO_ECUDA;
  void* args[] = {&A, &m, &n, &V, &tau, &beta, &frob2, &flags, &epoch, &err};
  cudaError_t e = cudaLaunchCooperativeKernel((void*)qr_coop_kernel, dim3(G), dim3(256), args, smem, L.stream);
  ++*L.launches;
  if (L.prof) L.prof->end(L.stream, pr);
  return e == cudaSuccess ? 0 : TEVO_ECUDA;
}

size_t qr64_wy_bytes(int n) {
  const size_t nblk = (size_t)(n + WY_NB - 1) / WY_NB;
  return 2 * nblk * WY_NB * WY_NB * sizeof(double2);
}

int qr64_form_q(const Launch& L, const z64* V_, const z64* tau_, int m, int n, z64* Q, long long sQr, long long sQc,
                void* wy) {
  if (m < n || n <= 0) return TEVO_ESHAPE;
  const size_t smem = sizeof(double2) * (size_t)m;
  if (smem > 200 * 1024) return TEVO_EUNSUPPORTED;
  static std::atomic<unsigned long long> attr{0};
  if (smem > 48 * 1024 && smem_attr_once(qr_wy_form_kernel, 200 * 1024, attr)) return TEVO_ECUDA;
  const double2* V = reinterpret_cast<const double2*>(V_);
  const double2* tau = reinterpret_cast<const double2*>(tau_);
  const int nblk = (n + WY_NB - 1) / WY_NB;
  double2* G = static_cast<double2*>(wy);
  double2* Tf = G + (size_t)nblk * WY_NB * WY_NB;
  // complex Householder Q formation: 8 (m n^2 - n^3 / 3) flops
  const double fflops = 8.0 * ((double)m * n * n - (double)n * n * n / 3.0);
  int pr = L.prof ? L.prof->begin(L.stream, TEVO_PROF_FORMQ, fflops, 32.0 * (double)m * n) : -1;
  if (nblk > 65535) return TEVO_ESHAPE;
  qr_wy_gram_kernel<<<dim3(nblk, WY_GRAM_SPLIT), 256, 0, L.stream>>>(V, m, n, G);
  qr_wy_t_kernel<<<nblk, 32, 0, L.stream>>>(tau, n, G, Tf);
  qr_wy_form_kernel<<<n, 512, smem, L.stream>>>(V, m, n, Tf, reinterpret_cast<double2*>(Q), sQr, sQc,
                                                std::min(n, L.num_sms));
  *L.launches += 3;
  if (L.prof) L.prof->end(L.stream, pr);
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int jacobi_top_columns(const Launch& L, z64* A_, int M, int N, int k, z64* out, void* ws, int* err) {
  if (M < 1 || N < 2 || (N & 1) || k < 1 || k > N) return TEVO_ESHAPE;
  double2* A = reinterpret_cast<double2*>(A_);
  unsigned int* bar = static_cast<unsigned int*>(ws);
  int* votes = reinterpret_cast<int*>(bar + 64);
  double* frob2 = reinterpret_cast<double*>(votes + JAC_MAX_SWEEPS + 64);
  double* part = frob2 + 8;
  double* nrm = part + FROB_BLOCKS;
  if (cudaMemsetAsync(ws, 0, sizeof(unsigned int) * (64 + JAC_MAX_SWEEPS + 64), L.stream) != cudaSuccess)
    return TEVO_ECUDA;
  int G = std::min(N / 2, L.num_sms);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_cols_kernel, 256, 0) != cudaSuccess ||
      per_sm * L.num_sms < G)
    return TEVO_EUNSUPPORTED;
  frob_partial_kernel<<<FROB_BLOCKS, 256, 0, L.stream>>>(A, (long long)M * N, part);
  sum_partials_kernel<<<1, 256, 0, L.stream>>>(part, FROB_BLOCKS, frob2);
  *L.launches += 2;
  int maxsw = JAC_MAX_SWEEPS;
  // pairs count as orthogonal below a few roundings of an M-term dot product
  double tol = std::max(JAC_TOL, 2.0 * std::sqrt((double)M) * 2.220446049250313e-16);
  const double* f2 = frob2;
  void* args[] = {&A, &M, &N, &maxsw, &tol, &f2, &bar, &votes, &err};
  if (cudaLaunchCooperativeKernel((void*)jacobi_cols_kernel, dim3(G), dim3(256), args, 0, L.stream) != cudaSuccess)
    return TEVO_ECUDA;
  const int nb = std::max(1, std::min((N * 32 + 255) / 256, 8 * L.num_sms));
  col_norms_kernel<<<nb, 256, 0, L.stream>>>(A, M, N, nrm);
  gather_top_kernel<<<N, 256, 0, L.stream>>>(A, M, N, nrm, k, reinterpret_cast<double2*>(out));
  *L.launches += 3;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

size_t jacobi_ws_bytes(int N) {
  return sizeof(unsigned int) * (64 + JAC_MAX_SWEEPS + 64) + sizeof(double) * (8 + FROB_BLOCKS + N + 64);
}

int qr64_extract_r(const Launch& L, const z64* A, const z64* beta, int m, int n, z64* R) {
  long long total = (long long)n * n;
  int blocks = int(std::min<long long>((total + 255) / 256, 4LL * L.num_sms));
  qr_extract_r_kernel<<<blocks, 256, 0, L.stream>>>(reinterpret_cast<const double2*>(A),
                                                    reinterpret_cast<const double2*>(beta), m, n,
                                                    reinterpret_cast<double2*>(R));
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

// ---------------------------------------------------------------------------
// layout and reduction helpers
// ---------------------------------------------------------------------------
namespace {

__global__ void mirror_kernel(const double2* in, double2* out, int na, int d, int nb) {
  long long total = (long long)na * d * nb;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    // idx enumerates out[b][s][a]
    int a = int(idx % na);
    long long t = idx / na;
    int s = int(t % d);
    int b = int(t / d);
    out[idx] = in[((long long)a * d + s) * nb + b];
  }
}

__global__ void copy2d_kernel(const double2* src, long long sr, long long sc, double2* dst, long long dr,
                              long long dc, int rows, int cols) {
  long long total = (long long)rows * cols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int r = int(idx / cols), c = int(idx % cols);
    dst[r * dr + c * dc] = src[r * sr + c * sc];
  }
}

__global__ void fill_kernel(double2* dst, long long n, double re, double im) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    dst[idx] = make_double2(re, im);
}

__global__ void eye_kernel(double2* dst, int n) {
  const long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    dst[idx] = make_double2(idx / n == idx % n ? 1.0 : 0.0, 0.0);
}

__global__ void normalize_kernel(double2* x, long long n, const double* nrm2, double* lognorm, int* flag) {
  const double s2 = *nrm2;
  const bool bad = !(s2 > 0.0) || !isfinite(s2);
  if (bad) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 1;
    return;
  }
  const double inv = 1.0 / sqrt(s2);
  if (blockIdx.x == 0 && threadIdx.x == 0) *lognorm += 0.5 * log(s2);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    double2 v = x[idx];
    x[idx] = make_double2(v.x * inv, v.y * inv);
  }
}

__global__ void dotu_partial_kernel(const double2* a, const double2* b, long long n, double* part) {
  __shared__ double red[64];
  double2 s = make_double2(0.0, 0.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s = cfma(a[i], b[i], s);
  double2 t = block_csum(s, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t.x;
    part[2 * blockIdx.x + 1] = t.y;
  }
}

__global__ void dotu_final_kernel(const double* part, int np, double2* out) {
  __shared__ double red[64];
  double2 s = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    s.x += part[2 * i];
    s.y += part[2 * i + 1];
  }
  double2 t = block_csum(s, red);
  if (threadIdx.x == 0) *out = t;
}

// one site's density in the mixed gauge with identity right transfers:
// part[blk][s][t] = sum over this block's (a0, a) of conj(A[a0][s][a]) Y[a0][t][a]
// for A, Y of shape [Dl][d][Dr] (Y = El A), d <= RHO_MAX_D; each of the d^2
// sums in block_csum's fixed order
constexpr int RHO_MAX_D = 4;
constexpr int RHO_BLOCKS = 64;
__global__ void rho_partial_kernel(const double2* A, const double2* Y, int Dl, int d, int Dr, double2* part) {
  __shared__ double red[64];
  double2 acc[RHO_MAX_D * RHO_MAX_D];
#pragma unroll
  for (int j = 0; j < RHO_MAX_D * RHO_MAX_D; ++j) acc[j] = make_double2(0.0, 0.0);
  const long long n = (long long)Dl * Dr;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long a0 = idx / Dr, a = idx % Dr;
    const double2* Ar = A + a0 * d * Dr + a;
    const double2* Yr = Y + a0 * d * Dr + a;
#pragma unroll
    for (int s = 0; s < RHO_MAX_D; ++s)
#pragma unroll
      for (int t = 0; t < RHO_MAX_D; ++t)
        if (s < d && t < d) acc[s * RHO_MAX_D + t] = cfma(cconj(Ar[(long long)s * Dr]), Yr[(long long)t * Dr],
                                                          acc[s * RHO_MAX_D + t]);
  }
#pragma unroll
  for (int s = 0; s < RHO_MAX_D; ++s)
#pragma unroll
    for (int t = 0; t < RHO_MAX_D; ++t)
      if (s < d && t < d) {  // uniform across the block
        const double2 v = block_csum(acc[s * RHO_MAX_D + t], red);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * d * d + s * d + t] = v;
      }
}

// vals[k][i] = sum_{s,t} O_k[s][t] rho_i[s][t], rho_i the blocks' partials of
// site i summed in block order (one thread per (k, i))
__global__ void rho_apply_kernel(const double2* part, int L, int d, const double2* ops, int nops, double2* vals) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nops * L) return;
  const int k = idx / L, i = idx % L;
  double2 v = make_double2(0.0, 0.0);
  for (int s = 0; s < d; ++s)
    for (int t = 0; t < d; ++t) {
      double2 r = make_double2(0.0, 0.0);
      for (int b = 0; b < RHO_BLOCKS; ++b) {
        const double2 p = part[((long long)i * RHO_BLOCKS + b) * d * d + s * d + t];
        r.x += p.x;
        r.y += p.y;
      }
      v = cfma(ops[(long long)k * d * d + s * d + t], r, v);
    }
  vals[idx] = v;
}

__global__ void rescale_kernel(double2* E, long long n, const double* nrm2, double* logacc) {
  const double s2 = *nrm2;
  if (!(s2 > 0.0) || !isfinite(s2)) return;
  const double inv = 1.0 / sqrt(s2);
  if (blockIdx.x == 0 && threadIdx.x == 0) *logacc += 0.5 * log(s2);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    double2 v = E[idx];
    E[idx] = make_double2(v.x * inv, v.y * inv);
  }
}

int grid_for(long long n, int num_sms) {
  long long b = (n + 255) / 256;
  long long cap = 8LL * num_sms;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return int(b);
}

}  // namespace

int mirror_site64(const Launch& L, const z64* in, z64* out, int na, int d, int nb) {
  long long total = (long long)na * d * nb;
  mirror_kernel<<<grid_for(total, L.num_sms), 256, 0, L.stream>>>(reinterpret_cast<const double2*>(in),
                                                                    reinterpret_cast<double2*>(out), na, d, nb);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int copy2d64(const Launch& L, const z64* src, long long sr, long long sc, z64* dst, long long dr, long long dc,
             int rows, int cols) {
  long long total = (long long)rows * cols;
  if (total <= 0) return 0;
  copy2d_kernel<<<grid_for(total, L.num_sms), 256, 0, L.stream>>>(reinterpret_cast<const double2*>(src), sr, sc,
                                                                   reinterpret_cast<double2*>(dst), dr, dc, rows,
                                                                   cols);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int fill64(const Launch& L, z64* dst, size_t n, double re, double im) {
  if (n == 0) return 0;
  fill_kernel<<<grid_for((long long)n, L.num_sms), 256, 0, L.stream>>>(reinterpret_cast<double2*>(dst),
                                                                       (long long)n, re, im);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int eye64(const Launch& L, z64* dst, int n) {
  if (n <= 0) return 0;
  eye_kernel<<<grid_for((long long)n * n, L.num_sms), 256, 0, L.stream>>>(reinterpret_cast<double2*>(dst), n);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int norm2_64(const Launch& L, const z64* x, size_t n, double* out, double* scratch) {
  frob_partial_kernel<<<FROB_BLOCKS, 256, 0, L.stream>>>(reinterpret_cast<const double2*>(x), (long long)n,
                                                         scratch);
  sum_partials_kernel<<<1, 256, 0, L.stream>>>(scratch, FROB_BLOCKS, out);
  *L.launches += 2;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int normalize64(const Launch& L, z64* x, size_t n, const double* nrm2, double* lognorm, int* flag) {
  normalize_kernel<<<grid_for((long long)n, L.num_sms), 256, 0, L.stream>>>(reinterpret_cast<double2*>(x),
                                                                             (long long)n, nrm2, lognorm, flag);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int dotu64(const Launch& L, const z64* a, const z64* b, size_t n, z64* out, double* scratch) {
  dotu_partial_kernel<<<FROB_BLOCKS, 256, 0, L.stream>>>(reinterpret_cast<const double2*>(a),
                                                         reinterpret_cast<const double2*>(b), (long long)n, scratch);
  dotu_final_kernel<<<1, 256, 0, L.stream>>>(scratch, FROB_BLOCKS, reinterpret_cast<double2*>(out));
  *L.launches += 2;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

size_t rho_part_count(int L, int d) { return (size_t)L * RHO_BLOCKS * d * d; }

int rho_partial64(const Launch& L, const z64* A, const z64* Y, int Dl, int d, int Dr, z64* part) {
  if (d < 1 || d > RHO_MAX_D) return TEVO_EUNSUPPORTED;
  rho_partial_kernel<<<RHO_BLOCKS, 256, 0, L.stream>>>(reinterpret_cast<const double2*>(A),
                                                      reinterpret_cast<const double2*>(Y), Dl, d, Dr,
                                                      reinterpret_cast<double2*>(part));
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int rho_apply64(const Launch& L, const z64* part, int nsites, int d, const z64* ops, int nops, z64* vals) {
  const int n = nops * nsites;
  rho_apply_kernel<<<(n + 127) / 128, 128, 0, L.stream>>>(reinterpret_cast<const double2*>(part), nsites, d,
                                                          reinterpret_cast<const double2*>(ops), nops,
                                                          reinterpret_cast<double2*>(vals));
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int rescale64(const Launch& L, z64* E, size_t n, double* logacc, double* scratch) {
  double* nrm2 = scratch + 2 * FROB_BLOCKS;
  frob_partial_kernel<<<FROB_BLOCKS, 256, 0, L.stream>>>(reinterpret_cast<const double2*>(E), (long long)n,
                                                         scratch);
  sum_partials_kernel<<<1, 256, 0, L.stream>>>(scratch, FROB_BLOCKS, nrm2);
  rescale_kernel<<<grid_for((long long)n, L.num_sms), 256, 0, L.stream>>>(reinterpret_cast<double2*>(E),
                                                                           (long long)n, nrm2, logacc);
  *L.launches += 3;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

}  // namespace tevo
