// Complex fp64 GEMM emulated on the bf16 tensor cores: the splitting form of the
// Ozaki scheme (error-free products of integer digit slices).
//
//   C[m][n] = sum_k A[m][k] * B[n][k]      (fp64 complex in, fp64 complex out)
//
// Every row r of an operand is scaled by a power of two 2^-e_r with
// max_k max(|Re|, |Im|) < 2^e_r, and the scaled row (entries in (-1, 1)) is cut
// into G digit slices
//   x = 2^e_r * sum_s alpha_s * 2^-(P + W s) + rest,   |alpha_s| <= 2^P,
// taken as the balanced base-2^W digits of x 2^-e_r rounded to a fixed-point
// integer of P + W (G - 1) fraction bits, P = 6, W = 7 bits per slice,
// |rest| <= 2^(e_r - W G). Scaling and slicing work on the bit patterns with
// integer operations; a row holding a NaN or an infinity gives NaN outputs.
// The digits are integers of at most 7 significant bits, so they are exact in
// bf16, their products (at most 2^12) are exact, and a sum of up to 4096 such
// products is an integer below 2^24: exact in the fp32 accumulator of the
// tensor core, whatever the order of summation.
//
// C is formed from the slice pairs (s, t) with s + t < G, grouped by g = s + t
// (all pairs of a group carry the weight 2^-(2P + W g)). One pass accumulates a
// group over at most 2048 / (g + 1) K-indices: 2 (g + 1) K <= 4096 terms, so
// the pass result is exact. The epilogue turns it into an integer and adds it,
// shifted left by its group's weight, to one of two 64-bit fixed-point sums per
// output entry (groups 0..3 and groups 4..7, the second in units 2^-28 of the
// first), so the sums are exact; after the last pass of a tile the entry is
// the exact 128-bit combination of the two, scaled by 2^(e_m + e_n) and rounded
// once to fp64. The only errors are the dropped terms (digits past slice G-1
// and pairs with s + t >= G), relative size about (G + 2) 2^-(W G) of
// max|A_m.| max|B_n.| K (G = 8: 56 bits), and that final rounding. No per-pass
// work uses the fp64 pipe, which on this part runs at about 1/1600 of the bf16
// MMA rate.
//
// The tensor-core schedule is that of the plain complex GEMM (k_tc.cu): a
// persistent CTA per SM, a TMA producer warp, one thread issuing tcgen05.mma,
// twelve epilogue warps (three per tensor-memory lane quarter), two tensor-memory
// accumulator buffers (a pass drains while the next accumulates). A stage holds
// the (re, im) planes of one A slice and the (-im, re, im) planes of one B slice
// for 32 K-indices. The accumulator of a 128 x 128 complex tile is one
// 128 x 256 fp32 block, Re in columns 0..127 and Im in 128..255, and each 16 K
// take two real MMAs of N = 256 whose B operands are two consecutive planes:
//   [Re | Im] += Ar [Br ; Bi]  and  [Re | Im] += Ai [-Bi ; Br].
// (Four N = 128 MMAs per 16 K ran the tensor pipe about 1.5x slower.)
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "tc_ptx.cuh"
#include "tevo_internal.h"
#include "tevo_tc.h"

namespace tevo {

namespace {

constexpr int OZ_P = 6;           // digits are integers in [-2^P, 2^P]
constexpr int OZ_W = 7;           // weight ratio between consecutive slices: 2^W
constexpr int OZ_MAX_SLICES = 8;  // (g + 1) * 256 <= 2048 keeps every pass below 2^24
// pass values of groups 0..3 are summed in one 64-bit fixed-point accumulator,
// those of groups 4..7 in a second one whose unit is 2^-28 of the first: every
// pass value then enters its sum shifted left (never right), so both sums are
// exact, and the entry is their exact 128-bit combination, rounded once
constexpr int OZ_HI_GROUPS = 4;
constexpr int OZ_LO_SHIFT = OZ_W * OZ_HI_GROUPS;
constexpr int OZ_TM = 128, OZ_TN = 128;
constexpr int OZ_KCB = 64;                 // bytes of K per stage row (32 bf16)
constexpr int OZ_KT_CHUNK = 8;             // K-tiles of 32 per exact chunk: 256 K-indices
constexpr int OZ_NSTAGE = 5;
constexpr int OZ_A_PLANES = 2;                  // per A slice: re, im
constexpr int OZ_B_PLANES = 3;                  // per B slice: -im, re, im
constexpr int OZ_A_BYTES = OZ_A_PLANES * OZ_TM * OZ_KCB;  // 16 KB
constexpr int OZ_B_BYTES = OZ_B_PLANES * OZ_TN * OZ_KCB;  // 24 KB
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr int OZ_SMEM_BYTES = OZ_NSTAGE * OZ_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
#ifndef OZ_EPILOGUE_WARPS
#define OZ_EPILOGUE_WARPS 12
#endif
// epilogue warps: one to four per tensor-memory lane quarter, each on a run of
// the tile's columns. Twelve (three per quarter, 128 registers a thread) keep
// 1.5x the fixed-point-sum loads of eight in flight and ran the kernel 2-9 %
// faster; sixteen spill at the 96 registers a thread they leave.
constexpr int OZ_EPI_WARPS = OZ_EPILOGUE_WARPS;
static_assert(OZ_EPI_WARPS % 4 == 0 && OZ_EPI_WARPS <= 16, "epilogue warps");
constexpr int OZ_THREADS = 32 * (2 + OZ_EPI_WARPS);
// one operand to cut into digit slices: element (r, k) of R x K at
// src[(r / R2) * sR1 + (r % R2) * sR + k * sK] (conjugated when conj), digit
// planes written to dst[p * plane_stride + r * row_pitch + k] (planes per
// slice: 2 = re, im; 3 = -im, re, im), the row maxima
// of the entries' exponent bounds to rowexp[r] (set to OZ_NONE before), the
// row exponents to exps[r]
struct OzSplit {
  const double2* src;
  long long sR, sK;
  int R, K;
  int conj;
  int G;
  __nv_bfloat16* dst;
  long long plane_stride, row_pitch;
  int* exps;
  int* rowexp;
  int R2;
  long long sR1;
  int planes;
};

__device__ __forceinline__ long long row_offset(const OzSplit& o, long long r) {
  return (r / o.R2) * o.sR1 + (r % o.R2) * o.sR;
}

struct OzArgs {
  int M, N, G;
  int k_tiles, nchunks, cps, splits;  // K-tiles of 32, exact chunks, chunks per split
  const int* ea;                      // row exponents of A (M) and of B (N)
  const int* eb;
  double2* C;  // output when splits == 1: (m, n) at m sCm + (n / N2) sCn1 + (n % N2) sCn
  long long sCm, sCn;
  int N2;
  long long sCn1;
  double2* part;  // [splits][M][N] when splits > 1
  longlong2* acc;  // fixed-point sums: [CTA][2][column][row], two sums of one 128 x 128 tile per CTA
  int base_shift;  // S unit: 2^-base_shift of a group-0 pass value
  int* err;
};

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// row exponent marking a row that holds a NaN or an infinity: its digits are
// zero and every output entry it touches is NaN
constexpr int OZ_NONFINITE = 0x7fff0000;
// "no entry yet" of the exponent maxima (the byte pattern 0x80 repeated, so a
// memset initialises it); far below any exponent of a finite double
constexpr int OZ_NONE = (int)0x80808080;

// exponent e with |v| < 2^e for the larger of |Re v|, |Im v| (from the binary64
// fields): OZ_NONE for zero, OZ_NONFINITE for a NaN or an infinity
__device__ __forceinline__ int exp_bound(double2 v) {
  const unsigned long long ax = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long ay = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long mx = ax > ay ? ax : ay;
  if (mx == 0) return OZ_NONE;
  const int E = (int)(mx >> 52);
  if (E == 0x7FF) return OZ_NONFINITE;
  return E == 0 ? -1022 : E - 1022;
}

// x * 2^(F - e) rounded to the nearest integer (ties to even), for |x| < 2^e:
// the common fixed point of a row's digits (F = P + W (G - 1) <= 55 bits)
__device__ __forceinline__ long long to_fixed(double x, int e, int F) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & ((1ull << 52) - 1ull);
  if (E == 0 && m == 0) return 0;
  if (E != 0) m |= 1ull << 52;
  const int sh = (E == 0 ? 1 : E) - 1075 - e + F;  // x = m 2^(E - 1075)
  unsigned long long X;
  if (sh >= 0) {
    X = m << sh;  // < 2^F since |x| < 2^e
  } else if (sh <= -64) {
    X = 0;
  } else {
    const int q = -sh;
    X = m >> q;
    const unsigned long long rem = m & ((1ull << q) - 1ull), half = 1ull << (q - 1);
    if (rem > half || (rem == half && (X & 1ull))) ++X;
  }
  return (b >> 63) ? -(long long)X : (long long)X;
}

// s * 2^e2 in fp64, rounded to nearest (ties to even), assembled from the
// binary64 fields with integer operations; results outside the normal range
// take the conversion instruction and an exact power-of-two scaling instead
#ifdef __CUDA_ARCH__
__noinline__
#endif
__host__ __device__ double fixed_to_f64(long long s, int e2) {
  if (s == 0) return 0.0;
  const unsigned long long neg = (unsigned long long)s >> 63;
  const unsigned long long u = neg ? 0ull - (unsigned long long)s : (unsigned long long)s;
#ifdef __CUDA_ARCH__
  const int nb = 64 - __clzll((long long)u);
#else
  const int nb = 64 - __builtin_clzll(u);
#endif
  const int ex = nb - 1 + e2;  // exponent of the leading bit
  if (ex < -1022 || ex > 1022) return ldexp((double)s, e2);
  unsigned long long q;
  int exq = ex;
  if (nb <= 53) {
    q = u << (53 - nb);
  } else {
    const int drop = nb - 53;  // 1..11 bits below the 53 kept
    q = u >> drop;
    const unsigned long long rem = u & ((1ull << drop) - 1ull), half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (q & 1ull))) {
      ++q;
      if (q >> 53) {
        q >>= 1;
        ++exq;
      }
    }
  }
  const unsigned long long bits = (neg << 63) | ((unsigned long long)(exq + 1023) << 52) | (q & ((1ull << 52) - 1ull));
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  std::memcpy(&d, &bits, sizeof(d));
  return d;
#endif
}

// (hi 2^64 + lo) * 2^e2 for a two's-complement 128-bit integer, rounded to the
// nearest fp64 (ties to even) from its leading 64 bits and a sticky bit for the
// rest; results outside the normal range take an exact power-of-two scaling of
// the rounded 53-bit significand
#ifdef __CUDA_ARCH__
__noinline__
#endif
__host__ __device__ double fixed128_to_f64(long long hi, unsigned long long lo, int e2) {
  const bool neg = hi < 0;
  unsigned long long uh = (unsigned long long)hi, ul = lo;
  if (neg) {
    ul = ~ul + 1ull;
    uh = ~uh + (ul == 0 ? 1ull : 0ull);
  }
  if (uh == 0 && ul == 0) return 0.0;
  int sh = 0;  // bits of the magnitude below its leading 64
  unsigned long long top = ul;
  bool sticky = false;
  if (uh != 0) {
#ifdef __CUDA_ARCH__
    sh = 64 - __clzll((long long)uh);
#else
    sh = 64 - __builtin_clzll(uh);
#endif
    top = sh == 64 ? uh : ((uh << (64 - sh)) | (ul >> sh));
    sticky = sh == 64 ? (ul != 0) : ((ul & ((1ull << sh) - 1ull)) != 0);
  }
#ifdef __CUDA_ARCH__
  const int nb = 64 - __clzll((long long)top);
#else
  const int nb = 64 - __builtin_clzll(top);
#endif
  unsigned long long q;
  int exq = nb - 1 + sh + e2;  // exponent of the leading bit
  if (nb <= 53) {
    q = top << (53 - nb);  // exact (sticky is set only when nb == 64)
  } else {
    const int drop = nb - 53;
    q = top >> drop;
    const unsigned long long rem = top & ((1ull << drop) - 1ull), half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (sticky || (q & 1ull)))) {
      ++q;
      if (q >> 53) {
        q >>= 1;
        ++exq;
      }
    }
  }
  if (exq < -1022 || exq > 1023) {
    const double r = ldexp((double)q, exq - 52);
    return neg ? -r : r;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(exq + 1023) << 52) |
                                  (q & ((1ull << 52) - 1ull));
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  std::memcpy(&d, &bits, sizeof(d));
  return d;
#endif
}

// the exact value S0 2^OZ_LO_SHIFT + S1 of the two fixed-point sums, times 2^e2
__device__ __forceinline__ double combine_to_f64(long long s0, long long s1, int e2) {
  // s0 2^28 as 128 bits, then + s1 sign-extended
  long long hi = s0 >> (64 - OZ_LO_SHIFT);
  unsigned long long lo = (unsigned long long)s0 << OZ_LO_SHIFT;
  const unsigned long long lo2 = lo + (unsigned long long)s1;
  hi += (s1 >> 63) + (lo2 < lo ? 1 : 0);
  return fixed128_to_f64(hi, lo2, e2);
}

// row maxima of the exponent bounds: a warp reduces one row over a
// segment of 256 K-indices (K contiguous or general strides) and merges it
// with atomicMax, so long rows are spread over many warps
__global__ void oz_rowmax_warp_kernel(OzSplit o, int nseg) {
  const int lane = threadIdx.x % 32;
  const long long nwarps = (long long)o.R * nseg;
  for (long long w = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < nwarps;
       w += (long long)gridDim.x * (blockDim.x / 32)) {
    const long long r = w / nseg;
    const int k0 = int(w % nseg) * 256;
    const double2* src = o.src + row_offset(o, r);
    // the segment's eight loads per lane issued together
    double2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + lane + 32 * j;
      v[j] = k < o.K ? src[(long long)k * o.sK] : make_double2(0.0, 0.0);
    }
    int mx = OZ_NONE;
#pragma unroll
    for (int j = 0; j < 8; ++j) mx = max(mx, exp_bound(v[j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0 && mx != OZ_NONE) atomicMax(o.rowexp + r, mx);
  }
}

// the same when rows are contiguous: a warp covers 32 consecutive rows (one per
// lane) over a segment of 64 K-indices
__global__ void oz_rowmax_lane_kernel(OzSplit o, int nseg) {
  const long long nrow32 = ((long long)o.R + 31) / 32;
  const long long nwarps = nrow32 * nseg;
  const int lane = threadIdx.x % 32;
  for (long long w = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < nwarps;
       w += (long long)gridDim.x * (blockDim.x / 32)) {
    const long long r = (w / nseg) * 32 + lane;
    const int k0 = int(w % nseg) * 64;
    if (r >= o.R) continue;
    const double2* src = o.src + row_offset(o, r);
    int mx = OZ_NONE;
    for (int k = k0; k < min(o.K, k0 + 64); ++k) mx = max(mx, exp_bound(src[(long long)k * o.sK]));
    if (mx != OZ_NONE) atomicMax(o.rowexp + r, mx);
  }
}

// balanced base-2^W digits of a fixed-point value X (|X| <= 2^F): with
// U = X + C, C = 2^P sum_s 2^q_s (q_s = W (G - 1 - s)), digit s is the W-bit
// field of U at q_s minus 2^P (the leading digit takes all bits above q_0), so
// every digit lies in [-2^P, 2^P] and sum_s digit_s 2^q_s = X exactly
__device__ __forceinline__ int digit_of(unsigned long long U, int s, int G) {
  const int q = OZ_W * (G - 1 - s);
  const unsigned long long f = s == 0 ? (U >> q) : ((U >> q) & ((1ull << OZ_W) - 1ull));
  const int d = (int)min(f, (unsigned long long)(2 << OZ_P)) - (1 << OZ_P);  // the min never binds for |X| <= 2^F
  return d < -(1 << OZ_P) ? -(1 << OZ_P) : d;
}

// the digit planes of two neighbouring entries v0, v1 = (r, k), (r, k + 1) of a
// row with exponent e (OZ_NONFINITE: zeros), written as one 4-byte bf16 pair
// per plane; digit_bf16 holds the bf16 of the integers -2^P .. 2^P
__device__ __forceinline__ void write_digit_pair(const OzSplit& o, long long r, int k, int e, double2 v0, double2 v1,
                                                 const __nv_bfloat16* digit_bf16) {
  const int F = OZ_P + OZ_W * (o.G - 1);
  const bool fin = e != OZ_NONFINITE;
  unsigned long long C = 0;
  for (int s = 0; s < o.G; ++s) C += (1ull << OZ_P) << (OZ_W * (o.G - 1 - s));
  const unsigned long long u0r = (unsigned long long)(fin ? to_fixed(v0.x, e, F) : 0) + C;
  const unsigned long long u0i = (unsigned long long)(fin ? to_fixed(v0.y, e, F) : 0) + C;
  const unsigned long long u1r = (unsigned long long)(fin ? to_fixed(v1.x, e, F) : 0) + C;
  const unsigned long long u1i = (unsigned long long)(fin ? to_fixed(v1.y, e, F) : 0) + C;
  __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(o.dst + r * o.row_pitch + k);
  const long long ps2 = o.plane_stride / 2;  // plane stride in bf16 pairs (even: rows are padded to 8)
  constexpr int H = 1 << OZ_P;
  for (int s = 0; s < o.G; ++s) {
    __nv_bfloat162 re, im;
    re.x = digit_bf16[digit_of(u0r, s, o.G) + H];
    re.y = digit_bf16[digit_of(u1r, s, o.G) + H];
    const int d0i = digit_of(u0i, s, o.G), d1i = digit_of(u1i, s, o.G);
    im.x = digit_bf16[d0i + H];
    im.y = digit_bf16[d1i + H];
    if (o.planes == 3) {
      __nv_bfloat162 nim;
      nim.x = digit_bf16[H - d0i];
      nim.y = digit_bf16[H - d1i];
      dst[(long long)(3 * s) * ps2] = nim;
      dst[(long long)(3 * s + 1) * ps2] = re;
      dst[(long long)(3 * s + 2) * ps2] = im;
    } else {
      dst[(long long)(2 * s) * ps2] = re;
      dst[(long long)(2 * s + 1) * ps2] = im;
    }
  }
}

// digit planes [planes G][R][row_pitch] (planes = 2: plane 2s = Re of slice s,
// 2s+1 = Im; planes = 3: 3s = -Im, 3s+1 = Re, 3s+2 = Im) of a 32-row x 64-K tile, staged in shared memory so that the fp64 reads (along the
// contiguous source index) are coalesced; each thread then forms the digits of
// two neighbouring K entries and writes them as one 4-byte bf16 pair per plane
template <bool ROWS_CONTIG>
__global__ void oz_slice_kernel(OzSplit o) {
  __shared__ double2 tile[32][65];
  __shared__ __nv_bfloat16 digit_bf16[2 * (1 << OZ_P) + 1];  // bf16 of the integers -2^P .. 2^P
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  for (int t = threadIdx.y * 32 + threadIdx.x; t <= 2 * (1 << OZ_P); t += 256)
    digit_bf16[t] = __float2bfloat16_rn((float)(t - (1 << OZ_P)));
  if (ROWS_CONTIG) {
    for (int kk = threadIdx.y; kk < 64; kk += 8) {
      const int r = r0 + threadIdx.x, k = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (r < o.R && k < o.K) v = o.src[row_offset(o, r) + (long long)k * o.sK];
      if (o.conj) v.y = -v.y;
      tile[threadIdx.x][kk] = v;
    }
  } else {
    for (int i = threadIdx.y; i < 32; i += 8)
      for (int h = 0; h < 64; h += 32) {
        const int r = r0 + i, k = k0 + h + threadIdx.x;
        double2 v = make_double2(0.0, 0.0);
        if (r < o.R && k < o.K) v = o.src[row_offset(o, r) + (long long)k * o.sK];
        if (o.conj) v.y = -v.y;
        tile[i][h + threadIdx.x] = v;
      }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + 2 * threadIdx.x;
    if (r >= o.R || k >= o.K) continue;
    const int er = o.rowexp[r];
    const int e = er == OZ_NONE ? 0 : er;  // a zero row
    if (k0 == 0 && threadIdx.x == 0) o.exps[r] = e;
    // entries past K are zero (tile padding), so the pair never needs a tail case
    write_digit_pair(o, r, k, e, tile[i][2 * threadIdx.x], tile[i][2 * threadIdx.x + 1], digit_bf16);
  }
}

// rows of at most OZ_FUSED_MAX_K entries: a block holds OZ_FUSED_ROWS(K) whole
// rows in shared memory, takes each row's exponent (a warp per row) and writes
// its digit planes, so the operand is read once and no exponent pass runs.
// The exponent and the digits are those of oz_rowmax_* and oz_slice_kernel.
constexpr int OZ_FUSED_MAX_K = 512;
// rows per block: about 32 KB of shared memory, so that several blocks share an SM
__host__ __device__ constexpr int oz_fused_rows(int K) { return K <= 64 ? 32 : K <= 128 ? 16 : K <= 256 ? 8 : 4; }
// shared memory of a block for K (rows of 64-padded K plus one, to spread the banks)
__host__ __device__ constexpr int oz_fused_smem(int K) { return oz_fused_rows(K) * ((K + 63) / 64 * 64 + 1) * 16; }
constexpr int OZ_FUSED_SMEM = 32 * 65 * 16;  // the largest of oz_fused_smem (K = 64): 32.5 KB
static_assert(oz_fused_smem(64) == OZ_FUSED_SMEM && oz_fused_smem(128) <= OZ_FUSED_SMEM &&
                  oz_fused_smem(256) <= OZ_FUSED_SMEM && oz_fused_smem(512) <= OZ_FUSED_SMEM,
              "fused slicing shared memory");

template <bool ROWS_CONTIG>
__global__ void __launch_bounds__(256) oz_slice_rows_kernel(OzSplit o) {
  extern __shared__ double2 rows[];  // [RB][Kc + 1]
  __shared__ __nv_bfloat16 digit_bf16[2 * (1 << OZ_P) + 1];
  __shared__ int s_e[32];
  const int RB = oz_fused_rows(o.K), Kc = (o.K + 63) / 64 * 64, ld = Kc + 1;
  const long long r0 = (long long)blockIdx.x * RB;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int t = tid; t <= 2 * (1 << OZ_P); t += 256) digit_bf16[t] = __float2bfloat16_rn((float)(t - (1 << OZ_P)));
  // consecutive threads read consecutive addresses: rows when rows are
  // contiguous, K otherwise; up to eight loads in flight per thread before
  // their shared-memory stores
  const int ntile = RB * Kc;
  for (int base = 0; base < ntile; base += 8 * 256) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * 256 + tid;
      const int i = ROWS_CONTIG ? idx % RB : idx / Kc, k = ROWS_CONTIG ? idx / RB : idx % Kc;
      const long long r = r0 + i;
      v[u] = make_double2(0.0, 0.0);
      if (idx < ntile && r < o.R && k < o.K) v[u] = o.src[row_offset(o, r) + (long long)k * o.sK];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * 256 + tid;
      const int i = ROWS_CONTIG ? idx % RB : idx / Kc, k = ROWS_CONTIG ? idx / RB : idx % Kc;
      if (o.conj) v[u].y = -v[u].y;
      if (idx < ntile) rows[i * ld + k] = v[u];
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < RB; i += 8) {
    int mx = OZ_NONE;
    for (int k = threadIdx.x; k < o.K; k += 32) mx = max(mx, exp_bound(rows[i * ld + k]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (threadIdx.x == 0) {
      const int e = mx == OZ_NONE ? 0 : mx;  // a zero row
      s_e[i] = e;
      if (r0 + i < o.R) o.exps[r0 + i] = e;
    }
  }
  __syncthreads();
  // digits: with fewer than eight rows, the warps of a row split its K
  const int wpr = RB >= 8 ? 1 : 8 / RB;
  for (int i = threadIdx.y / wpr; i < RB; i += 8 / wpr) {
    const long long r = r0 + i;
    if (r >= o.R) continue;
    for (int k = 2 * threadIdx.x + 64 * (threadIdx.y % wpr); k < o.K; k += 64 * wpr)
      write_digit_pair(o, r, k, s_e[i], rows[i * ld + k], rows[i * ld + k + 1], digit_bf16);
  }
}

// fixed-order sum of the fp64 split partials into the strided output
__global__ void oz_reduce_kernel(const double2* P, int splits, int M, int N, double2* C, long long sCm,
                                 long long sCn, int N2, long long sCn1) {
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = int(idx / N), n = int(idx % N);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
      const double2 v = P[((long long)s * M + m) * N + n];
      re += v.x;
      im += v.y;
    }
    C[m * sCm + (long long)(n / N2) * sCn1 + (long long)(n % N2) * sCn] = make_double2(re, im);
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OZ_NSTAGE * OZ_STAGE_BYTES);
  // barriers: full[NSTAGE], empty[NSTAGE], tfull[2], tempty[2]; then the TMEM address slot
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_NSTAGE + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + OZ_NSTAGE);
  const uint32_t tfull0 = smem_u32(bars + 2 * OZ_NSTAGE), tempty0 = smem_u32(bars + 2 * OZ_NSTAGE + 2);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  const int mt = (a.M + OZ_TM - 1) / OZ_TM, nt = (a.N + OZ_TN - 1) / OZ_TN;
  // a unit is one row tile x one column tile x one split
  const int nunits = mt * nt * a.splits;
  const int cid = blockIdx.x, ncl = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_NSTAGE; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, OZ_EPI_WARPS);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // unit u -> (split z, row tile, column tile) and its chunk range [c0, c1)
  // the shorter tile dimension runs fastest, so CTAs that run together share
  // the tiles of the longer operand (read once from DRAM, then from L2)
  auto unit_of = [&](int u, int& m0, int& n0, int& c0, int& c1) {
    const int z = u / (mt * nt), r = u % (mt * nt);
    m0 = (mt <= nt ? r % mt : r / nt) * OZ_TM;
    n0 = (mt <= nt ? r / mt : r % nt) * OZ_TN;
    c0 = z * a.cps;
    c1 = min(a.nchunks, c0 + a.cps);
    return z;
  };
  // a unit covers the K-tiles [c0 * OZ_KT_CHUNK, min(c1 * OZ_KT_CHUNK, k_tiles));
  // a pass of group g spans at most 64 / (g + 1) K-tiles of 32, the longest
  // for which its 2 (g + 1) K products per entry stay exact in fp32 (so the
  // low groups, with little MMA work per K, need fewer passes)
  auto unit_tiles = [&](int c0, int c1, int& t0, int& t1) {
    t0 = c0 * OZ_KT_CHUNK;
    t1 = min(a.k_tiles, c1 * OZ_KT_CHUNK);
  };
  auto pass_len = [&](int g) { return (2048 / 32) / (g + 1); };

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      long long q = 0;  // stage ring counter
      bool ok = true;
      for (int u = cid; u < nunits && ok; u += ncl) {
        int m0, n0, c0, c1;
        unit_of(u, m0, n0, c0, c1);
        int t0, t1;
        unit_tiles(c0, c1, t0, t1);
        for (int g = 0; g < a.G && ok; ++g)
          for (int p0 = t0; p0 < t1 && ok; p0 += pass_len(g))
            for (int kt = p0; kt < min(t1, p0 + pass_len(g)) && ok; ++kt)
              for (int s = 0; s <= g; ++s, ++q) {
                const int st = int(q % OZ_NSTAGE);
                if (!mbar_wait(empty0 + 8 * st, (uint32_t(q / OZ_NSTAGE) & 1u) ^ 1u, a.err, 1)) {
                  ok = false;
                  break;
                }
                const uint32_t fb = full0 + 8 * st;
                mbar_expect_tx(fb, OZ_STAGE_BYTES);
                uint8_t* sp = smem + st * OZ_STAGE_BYTES;
                tma_load_4d(smem_u32(sp), &tmA, kt * 32, 0, m0, OZ_A_PLANES * s, fb);
                tma_load_4d(smem_u32(sp + OZ_A_BYTES), &tmB, kt * 32, 0, n0, OZ_B_PLANES * (g - s), fb);
              }
      }
      // do not leave while copies are in flight
      for (long long r = (q > OZ_NSTAGE ? q - OZ_NSTAGE : 0); r < q; ++r)
        mbar_wait(full0 + 8 * int(r % OZ_NSTAGE), uint32_t(r / OZ_NSTAGE) & 1u, a.err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // instruction descriptor: fp32 accumulate, bf16 A and B, K-major, M = 128,
      // N = 256 (the Re and Im column halves of the tile's accumulator)
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * OZ_TN) >> 3) << 17) |
                             ((uint32_t)(OZ_TM >> 4) << 24);
      const uint64_t plane_a = (uint64_t)((OZ_TM * OZ_KCB) >> 4), plane_b = (uint64_t)((OZ_TN * OZ_KCB) >> 4);
      long long q = 0;
      int i = 0;  // pass counter
      bool ok = true;
      for (int u = cid; u < nunits && ok; u += ncl) {
        int m0, n0, c0, c1;
        unit_of(u, m0, n0, c0, c1);
        int t0, t1;
        unit_tiles(c0, c1, t0, t1);
        for (int g = 0; g < a.G && ok; ++g)
          for (int p0 = t0; p0 < t1 && ok; p0 += pass_len(g), ++i) {
            const int kt0 = p0, kt1 = min(t1, p0 + pass_len(g));
            const int b = i & 1;
            if (!mbar_wait(tempty0 + 8 * b, (uint32_t(i >> 1) & 1u) ^ 1u, a.err, 5)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + (uint32_t)(b * 2 * OZ_TN);  // [Re | Im], 256 columns
            bool first = true;
            for (int kt = kt0; kt < kt1 && ok; ++kt)
              for (int s = 0; s <= g; ++s, ++q) {
                const int st = int(q % OZ_NSTAGE);
                if (!mbar_wait(full0 + 8 * st, uint32_t(q / OZ_NSTAGE) & 1u, a.err, 3)) {
                  ok = false;
                  break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_u32(smem + st * OZ_STAGE_BYTES);
                // B planes in the stage: 0 = -Bi, 1 = Br, 2 = Bi
                const uint64_t ar = sdesc(sa), bn = sdesc(sa + OZ_A_BYTES);
#pragma unroll
                for (int ks = 0; ks < OZ_KCB / 32; ++ks) {
                  const uint64_t o = (uint64_t)((ks * 32) >> 4);
                  const uint32_t acc = first ? 0u : 1u;
                  mma<TC_BF16>(dacc, ar + o, bn + plane_b + o, idesc, acc);  // [Re | Im]  = Ar [Br ; Bi]
                  mma<TC_BF16>(dacc, ar + plane_a + o, bn + o, idesc, 1u);   // [Re | Im] += Ai [-Bi ; Br]
                  first = false;
                }
                mma_commit(empty0 + 8 * st);
              }
            mma_commit(tfull0 + 8 * b);
          }
      }
    }
  } else {
    // epilogue: warps 2..; warp w owns tensor-memory lane quarter w % 4 and a
    // run of the tile's columns. A pass value is an exact integer held in fp32; the
    // passes of a unit are summed with integer operations only, groups 0..3 in
    // the 64-bit fixed-point accumulator S0 and groups 4..7 in S1 (unit 2^-28 of
    // S0's), both exact. They live in this CTA's slice of the workspace, laid
    // out [column][row] so that a warp touches 32 consecutive rows, and the entry
    // is converted to fp64 once, after the unit's last pass.
    const int qw = warp % 4;
    // this warp's columns: the tile's 128 split over the warps of a lane quarter
    // in runs of 16 (twelve warps: 48, 48, 32)
    const int nq = OZ_EPI_WARPS / 4, run = (warp - 2) / 4;
    const int per = ((OZ_TN / 16 + nq - 1) / nq) * 16;
    const int c_lo = min(OZ_TN, run * per);
    const int c_hi = min(OZ_TN, c_lo + per);
    const int row = qw * 32 + lane;
    longlong2* S0 = a.acc + (size_t)blockIdx.x * 2 * OZ_TM * OZ_TN + row;
    longlong2* S1 = S0 + OZ_TM * OZ_TN;
    int i = 0;
    bool ok = true;
    for (int u = cid; u < nunits && ok; u += ncl) {
      int m0, n0, c0, c1;
      const int z = unit_of(u, m0, n0, c0, c1);
      const int m = m0 + row;
      const int em = m < a.M ? a.ea[m] : 0;
      int t0, t1;
      unit_tiles(c0, c1, t0, t1);
      for (int g = 0; g < a.G && ok; ++g)
        for (int p0 = t0; p0 < t1; p0 += pass_len(g), ++i) {
          const int b = i & 1;
          if (!mbar_wait(tfull0 + 8 * b, uint32_t(i >> 1) & 1u, a.err, 4)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int h = g / OZ_HI_GROUPS;  // accumulator of this group
          longlong2* S = h ? S1 : S0;
          const bool first = (g == OZ_HI_GROUPS * h && p0 == t0), last = (g == a.G - 1 && p0 + pass_len(g) >= t1);
          // weight of this group in its sum: 2^shift units of the pass value,
          // shift = base_shift + 28 h - W g >= base_shift - 21 >= 0
          const int shift = a.base_shift + OZ_LO_SHIFT * h - OZ_W * g;
          const uint32_t trow = tmem + (uint32_t)(b * 2 * OZ_TN) + ((uint32_t)(qw * 32) << 16);
          for (int cc = c_lo; cc < c_hi; cc += 16) {
            uint32_t rr[16], ri[16];
            tmem_ld16(trow + cc, rr);
            tmem_ld16(trow + OZ_TN + cc, ri);
            // the 16 previous sums (independent loads in flight together)
            longlong2 old[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) old[j] = first ? make_longlong2(0, 0) : S[(size_t)(cc + j) * OZ_TM];
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const long long vr = (long long)__float2int_rn(__uint_as_float(rr[j]));
              const long long vi = (long long)__float2int_rn(__uint_as_float(ri[j]));
              S[(size_t)(cc + j) * OZ_TM] = make_longlong2(vr * (1LL << shift) + old[j].x, vi * (1LL << shift) + old[j].y);
            }
          }
          // this warp is done reading the buffer: hand it back to the MMA warp
          // (before the conversion below, which reads only the sums)
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty0 + 8 * b);
          if (last) {
            // the unit's entries of this lane's row: exact sums to fp64, once
            for (int col = c_lo; col < c_hi; ++col) {
              const int n = n0 + col;
              if (m >= a.M || n >= a.N) continue;
              double2* dst = a.splits == 1 ? a.C + (long long)m * a.sCm + (long long)(n / a.N2) * a.sCn1 +
                                                 (long long)(n % a.N2) * a.sCn
                                           : a.part + ((long long)z * a.M + m) * (long long)a.N + n;
              const int en = a.eb[n];
              if (em == OZ_NONFINITE || en == OZ_NONFINITE) {
                *dst = make_double2(__longlong_as_double(0x7FF8000000000000LL),
                                    __longlong_as_double(0x7FF8000000000000LL));
              } else if (h == 0) {
                const longlong2 v = S0[(size_t)col * OZ_TM];
                const int e2 = em + en - 2 * OZ_P - a.base_shift;
                *dst = make_double2(fixed_to_f64(v.x, e2), fixed_to_f64(v.y, e2));
              } else {
                const longlong2 hi = S0[(size_t)col * OZ_TM], lo = S1[(size_t)col * OZ_TM];
                const int e2 = em + en - 2 * OZ_P - a.base_shift - OZ_LO_SHIFT;
                *dst = make_double2(combine_to_f64(hi.x, lo.x, e2), combine_to_f64(hi.y, lo.y, e2));
              }
            }
          }
        }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }
inline long long pad8(long long x) { return (x + 7) / 8 * 8; }

int grid_of(long long n, int per_block, int sms) {
  long long b = (n + per_block - 1) / per_block;
  if (b > 16LL * sms) b = 16LL * sms;
  return int(b < 1 ? 1 : b);
}

struct OzPlan {
  int k_tiles, nchunks, cps, splits, grid, base_shift;
  size_t a_bytes, b_bytes, e_bytes, p_bytes, s_bytes;
  size_t total() const { return a_bytes + b_bytes + e_bytes + p_bytes + s_bytes; }
};

OzPlan plan(int M, int N, int K, int G, int num_sms) {
  OzPlan p{};
  p.k_tiles = (K + 31) / 32;
  p.nchunks = (p.k_tiles + OZ_KT_CHUNK - 1) / OZ_KT_CHUNK;
  const long long tiles = (long long)((M + OZ_TM - 1) / OZ_TM) * ((N + OZ_TN - 1) / OZ_TN);
  int splits = (int)std::max<long long>(1, std::min<long long>((num_sms + tiles - 1) / tiles, p.nchunks));
  splits = std::min(splits, 64);
  p.cps = (p.nchunks + splits - 1) / splits;
  p.splits = (p.nchunks + p.cps - 1) / p.cps;
  const long long kp = pad8(K);
  p.a_bytes = al256((size_t)OZ_A_PLANES * G * M * kp * 2);
  p.b_bytes = al256((size_t)OZ_B_PLANES * G * N * kp * 2);
  p.e_bytes = al256((size_t)(M + N) * 2 * sizeof(int));
  p.p_bytes = p.splits > 1 ? al256((size_t)p.splits * M * N * 16) : 0;
  // persistent grid: one CTA per SM at most
  const long long units = (long long)((M + OZ_TM - 1) / OZ_TM) * ((N + OZ_TN - 1) / OZ_TN) * p.splits;
  p.grid = (int)std::max<long long>(1, std::min<long long>(units, (long long)num_sms));
  p.s_bytes = al256((size_t)p.grid * 2 * OZ_TM * OZ_TN * sizeof(longlong2));
  // |pass value| <= 2^24 and sum_g 2^-W g < 1.008: cps chunks stay below
  // 2^(base_shift + 24 + log2 cps + 0.02) <= 2^62.02 < 2^63
  int lg = 0;
  while ((1 << lg) < p.cps) ++lg;
  p.base_shift = 38 - lg;
  return p;
}

int split_operand(const Launch& L, const OzSplit& o) {
  const bool rows_contig = o.sR == 1 && o.sK != 1;
  if (o.K <= OZ_FUSED_MAX_K) {
    static std::atomic<unsigned long long> attr_t{0}, attr_f{0};
    if (smem_attr_once(oz_slice_rows_kernel<true>, OZ_FUSED_SMEM, attr_t) ||
        smem_attr_once(oz_slice_rows_kernel<false>, OZ_FUSED_SMEM, attr_f))
      return TEVO_ECUDA;
    const long long nb = ((long long)o.R + oz_fused_rows(o.K) - 1) / oz_fused_rows(o.K);
    if (nb > (1LL << 31) - 1) return TEVO_ESHAPE;
    const dim3 block(32, 8);
    if (rows_contig)
      oz_slice_rows_kernel<true><<<(unsigned)nb, block, oz_fused_smem(o.K), L.stream>>>(o);
    else
      oz_slice_rows_kernel<false><<<(unsigned)nb, block, oz_fused_smem(o.K), L.stream>>>(o);
    ++*L.launches;
    return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
  }
  if (cudaMemsetAsync(o.rowexp, 0x80, sizeof(int) * (size_t)o.R, L.stream) != cudaSuccess) return TEVO_ECUDA;
  if (rows_contig) {
    const int nseg = (o.K + 63) / 64;
    oz_rowmax_lane_kernel<<<grid_of(((long long)o.R + 31) / 32 * nseg * 32, 256, L.num_sms), 256, 0, L.stream>>>(o, nseg);
  } else {
    const int nseg = (o.K + 255) / 256;
    oz_rowmax_warp_kernel<<<grid_of((long long)o.R * nseg * 32, 256, L.num_sms), 256, 0, L.stream>>>(o, nseg);
  }
  ++*L.launches;
  if ((o.R + 31) / 32 > 65535) return TEVO_ESHAPE;
  dim3 grid((o.K + 63) / 64, (o.R + 31) / 32), block(32, 8);
  if (rows_contig)
    oz_slice_kernel<true><<<grid, block, 0, L.stream>>>(o);
  else
    oz_slice_kernel<false><<<grid, block, 0, L.stream>>>(o);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

}  // namespace

int oz_max_slices() { return OZ_MAX_SLICES; }

// a batch with a shared A operand is one GEMM over the batch-extended N
static long long total_n(const GemmDesc& g) { return (long long)g.N * std::max(1, g.batch); }

size_t ozgemm64_workspace(const GemmDesc& g, int slices, int num_sms) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || slices < 1 || slices > OZ_MAX_SLICES) return 0;
  if (g.batch > 1 && g.sAb != 0) return 0;
  if (total_n(g) > (1LL << 30)) return 0;
  const OzPlan p = plan(g.M, (int)total_n(g), g.K, slices, num_sms);
  return p.total();
}

int ozgemm64(const Launch& L, const GemmDesc& g, int slices, void* ws, size_t ws_bytes, int* err) {
  if (g.batch < 1 || (g.batch > 1 && g.sAb != 0) || g.conjB || g.alpha_re != 1.0 || g.alpha_im != 0.0 ||
      g.beta_re != 0.0 || g.beta_im != 0.0 || total_n(g) > (1LL << 30))
    return TEVO_EUNSUPPORTED;
  const int Nt = (int)total_n(g);
  if (slices < 1 || slices > OZ_MAX_SLICES) return TEVO_EINVAL;
  if (g.M <= 0 || g.N <= 0) return 0;
  if (g.K <= 0 || g.K > (1 << 25)) return TEVO_EUNSUPPORTED;  // keeps every accumulator shift >= 0
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr_once(oz_gemm_kernel, OZ_SMEM_BYTES, attr_done)) return TEVO_ECUDA;
  const OzPlan p = plan(g.M, Nt, g.K, slices, L.num_sms);
  if (!ws || !err || ws_bytes < p.total()) return TEVO_ESHAPE;
  char* w = static_cast<char*>(ws);
  __nv_bfloat16* da = reinterpret_cast<__nv_bfloat16*>(w);
  w += p.a_bytes;
  __nv_bfloat16* db = reinterpret_cast<__nv_bfloat16*>(w);
  w += p.b_bytes;
  int* mxa = reinterpret_cast<int*>(w);
  int* mxb = mxa + g.M;
  int* ea = mxb + Nt;
  int* eb = ea + g.M;
  w += p.e_bytes;
  double2* part = p.splits > 1 ? reinterpret_cast<double2*>(w) : nullptr;
  w += p.p_bytes;
  longlong2* acc = reinterpret_cast<longlong2*>(w);
  const long long kp = pad8(g.K);
  // A(m, k) at A + m sAm + k sAk; B(k, n) at B + k sBk + n sBn, read as rows n
  OzSplit sa{static_cast<const double2*>(g.A), g.sAm, g.sAk, g.M, g.K, g.conjA, slices, da, (long long)g.M * kp, kp,
             ea, mxa, g.M, 0, OZ_A_PLANES};
  // rows of B: (batch b, n) at b sBb + n sBn
  OzSplit sb{static_cast<const double2*>(g.B), g.sBn, g.sBk, Nt, g.K, 0, slices, db, (long long)Nt * kp, kp, eb,
             mxb, g.N, g.sBb, OZ_B_PLANES};
  const int pr_split = L.prof ? L.prof->begin(L.stream, TEVO_PROF_OZSPLIT, 0.0,
                                              ((16.0 + 4.0 * slices) * g.M + (16.0 + 6.0 * slices) * Nt) * g.K)
                              : -1;
  int e = split_operand(L, sa);
  if (!e) e = split_operand(L, sb);
  if (L.prof) L.prof->end(L.stream, pr_split);
  if (e) return e;

  TcOperand oa{da, 2, OZ_A_PLANES * slices, (long long)g.M * kp, g.M, kp, g.K, 1, kp};
  TcOperand ob{db, 2, OZ_B_PLANES * slices, (long long)Nt * kp, Nt, kp, g.K, 1, kp};
  CUtensorMap ma, mb;
  e = tc_make_map(&ma, oa, OZ_TM, OZ_A_PLANES);
  if (!e) e = tc_make_map(&mb, ob, OZ_TN, OZ_B_PLANES);
  if (e) return e;
  OzArgs a;
  std::memset(&a, 0, sizeof(a));
  a.M = g.M;
  a.N = Nt;
  a.G = slices;
  a.k_tiles = p.k_tiles;
  a.nchunks = p.nchunks;
  a.cps = p.cps;
  a.splits = p.splits;
  a.ea = ea;
  a.eb = eb;
  a.C = static_cast<double2*>(g.C);
  a.sCm = g.sCm;
  a.sCn = g.sCn;
  a.N2 = g.N;
  a.sCn1 = g.sCb;
  a.part = part;
  a.acc = acc;
  a.base_shift = p.base_shift;
  a.err = err;
  const long long units = (long long)((g.M + OZ_TM - 1) / OZ_TM) * ((Nt + OZ_TN - 1) / OZ_TN) * p.splits;
  if (units > (1LL << 30)) return TEVO_ESHAPE;
  const double useful = 8.0 * (double)g.M * Nt * g.K;
  const int pr = L.prof ? L.prof->begin(L.stream, TEVO_PROF_GEMMOZ, useful,
                                        16.0 * ((double)g.M * g.K + (double)Nt * g.K + (double)g.M * Nt))
                        : -1;
  oz_gemm_kernel<<<p.grid, OZ_THREADS, OZ_SMEM_BYTES, L.stream>>>(ma, mb, a);
  if (cudaGetLastError() != cudaSuccess) return TEVO_ECUDA;
  ++*L.launches;
  if (p.splits > 1) {
    oz_reduce_kernel<<<grid_of((long long)g.M * Nt, 256, L.num_sms), 256, 0, L.stream>>>(
        part, p.splits, g.M, Nt, static_cast<double2*>(g.C), g.sCm, g.sCn, g.N, g.sCb);
    ++*L.launches;
  }
  if (L.prof) L.prof->end(L.stream, pr);
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

}  // namespace tevo
