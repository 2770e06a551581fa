// Tensor-core complex GEMM for sm_103a: tcgen05.mma with accumulators in tensor
// memory, operands staged in shared memory by TMA (cp.async.bulk.tensor), one
// elected thread issuing the MMAs, mbarrier pipeline between the TMA producer
// warp and the MMA warp.
//
//   C[m][n] = sum_k A[m][k] * B[n][k]          (complex, both operands K-major)
//
// A complex operand is stored as "planes" of a real type: for the split forms
// (bf16x3, tf32x3) the planes are re_hi, re_lo, im_hi, im_lo with x = hi + lo;
// for plain tf32 they are re, im. A product of planes is one real MMA, so one
// complex K-step issues
//   Cr += Ar.Br - Ai.Bi,  Ci += Ar.Bi + Ai.Br
// per pair of split terms (hi.hi + hi.lo + lo.hi for the split forms: 12 MMAs;
// 4 MMAs for plain tf32), the minus sign through the negate-A bit of the
// instruction descriptor. Accumulation is fp32 in tensor memory.
//
// Each operand is a 4-D tensor [k_in, k_out, rows, planes] (k_in innermost).
// The K loop runs over (k_out, k_in chunk) pairs, so a reduction index that
// is itself two tensor modes with a padded inner mode (an environment's
// (w, psi) legs) is read through TMA bounds checks instead of padding.
//
// Persistent kernel: one CTA per SM walks the tiles (128 x 128 complex outputs,
// split-K chunks included) in a static round-robin order. Tensor memory holds
// two accumulator buffers (Cr, Ci of 128 columns each), so the epilogue warps
// drain tile i while the MMA warp accumulates tile i+1; the TMA producer runs
// ahead across tiles through a 3-stage ring of 64 KB stages (K chunk = 64 bytes
// per row: 32 bf16 / 16 fp32, 64B swizzle).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "tc_ptx.cuh"
#include "tevo_tc.h"

namespace tevo {

namespace {

constexpr int TM = 128, TN = 128;
constexpr int KCB = 64;  // bytes of K per stage row
constexpr int NSTAGE = 3;
constexpr int A_BYTES = 4 * TM * KCB;  // 32 KB (4 planes max)
constexpr int B_BYTES = 4 * TN * KCB;  // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int TC_THREADS = 192;

// self-test of the bounded wait: one thread waits on a barrier that nothing
// completes; the wait gives up after limit_ns and records `code`
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, err, 7, limit_ns);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// write one complex value into the planes of an output map
__device__ __forceinline__ void put(const TcOutMap& o, int fmt, long long off, float re, float im) {
  if (fmt == TC_BF16) {
    __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(o.base) + off;
    __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
    p[0] = rh;
    p[o.plane_stride] = __float2bfloat16_rn(re - __bfloat162float(rh));
    p[2 * o.plane_stride] = ih;
    p[3 * o.plane_stride] = __float2bfloat16_rn(im - __bfloat162float(ih));
  } else if (fmt == TC_TF32X3) {
    float* p = reinterpret_cast<float*>(o.base) + off;
    float rh = tf32_round(re), ih = tf32_round(im);
    p[0] = rh;
    p[o.plane_stride] = tf32_round(re - rh);
    p[2 * o.plane_stride] = ih;
    p[3 * o.plane_stride] = tf32_round(im - ih);
  } else {
    float* p = reinterpret_cast<float*>(o.base) + off;
    p[0] = tf32_round(re);
    p[o.plane_stride] = tf32_round(im);
  }
}

// 32 consecutive complex values of one row into every plane with 16-byte stores
__device__ __forceinline__ void put_row32(const TcOutMap& o, int fmt, long long off, const uint32_t* rr,
                                          const uint32_t* ri) {
  if (fmt == TC_BF16) {
    uint32_t h[4][16];
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      float r0 = __uint_as_float(rr[j]), r1 = __uint_as_float(rr[j + 1]);
      float i0 = __uint_as_float(ri[j]), i1 = __uint_as_float(ri[j + 1]);
      __nv_bfloat16 rh0 = __float2bfloat16_rn(r0), rh1 = __float2bfloat16_rn(r1);
      __nv_bfloat16 ih0 = __float2bfloat16_rn(i0), ih1 = __float2bfloat16_rn(i1);
      __nv_bfloat16 rl0 = __float2bfloat16_rn(r0 - __bfloat162float(rh0));
      __nv_bfloat16 rl1 = __float2bfloat16_rn(r1 - __bfloat162float(rh1));
      __nv_bfloat16 il0 = __float2bfloat16_rn(i0 - __bfloat162float(ih0));
      __nv_bfloat16 il1 = __float2bfloat16_rn(i1 - __bfloat162float(ih1));
      h[0][j / 2] = (uint32_t)__bfloat16_as_ushort(rh0) | ((uint32_t)__bfloat16_as_ushort(rh1) << 16);
      h[1][j / 2] = (uint32_t)__bfloat16_as_ushort(rl0) | ((uint32_t)__bfloat16_as_ushort(rl1) << 16);
      h[2][j / 2] = (uint32_t)__bfloat16_as_ushort(ih0) | ((uint32_t)__bfloat16_as_ushort(ih1) << 16);
      h[3][j / 2] = (uint32_t)__bfloat16_as_ushort(il0) | ((uint32_t)__bfloat16_as_ushort(il1) << 16);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(o.base) + off + p * o.plane_stride);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_uint4(h[p][4 * q], h[p][4 * q + 1], h[p][4 * q + 2], h[p][4 * q + 3]);
    }
  } else if (fmt == TC_TF32X3) {
    float* base = reinterpret_cast<float*>(o.base) + off;
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      float4 a0, a1, a2, a3;
      float* v0 = &a0.x;
      float* v1 = &a1.x;
      float* v2 = &a2.x;
      float* v3 = &a3.x;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float r = __uint_as_float(rr[j + t]), im = __uint_as_float(ri[j + t]);
        float rh = tf32_round(r), ih = tf32_round(im);
        v0[t] = rh;
        v1[t] = tf32_round(r - rh);
        v2[t] = ih;
        v3[t] = tf32_round(im - ih);
      }
      *reinterpret_cast<float4*>(base + j) = a0;
      *reinterpret_cast<float4*>(base + o.plane_stride + j) = a1;
      *reinterpret_cast<float4*>(base + 2 * o.plane_stride + j) = a2;
      *reinterpret_cast<float4*>(base + 3 * o.plane_stride + j) = a3;
    }
  } else {
    float* base = reinterpret_cast<float*>(o.base) + off;
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      *reinterpret_cast<float4*>(base + j) =
          make_float4(tf32_round(__uint_as_float(rr[j])), tf32_round(__uint_as_float(rr[j + 1])),
                      tf32_round(__uint_as_float(rr[j + 2])), tf32_round(__uint_as_float(rr[j + 3])));
      *reinterpret_cast<float4*>(base + o.plane_stride + j) =
          make_float4(tf32_round(__uint_as_float(ri[j])), tf32_round(__uint_as_float(ri[j + 1])),
                      tf32_round(__uint_as_float(ri[j + 2])), tf32_round(__uint_as_float(ri[j + 3])));
    }
  }
}

// batched transpose of plane-format matrices: dst(c, r) <- src(r, c), tile 32 x 32
template <typename T>
__global__ void transpose_planes_kernel(TcTranspose t) {
  __shared__ T tile[32][33];
  const int nb = t.batch;
  const int z = blockIdx.z;
  const int plane = z / nb, b = z % nb;
  const T* src = reinterpret_cast<const T*>(t.src) + plane * t.src_plane + (long long)(b / t.B2) * t.sb1 +
                 (long long)(b % t.B2) * t.sb2;
  T* dst = reinterpret_cast<T*>(t.dst) + plane * t.dst_plane + (long long)(b / t.B2) * t.db1 +
           (long long)(b % t.B2) * t.db2;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < t.R && c < t.C) tile[k][threadIdx.x] = src[(long long)r * t.s_r + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < t.R && c < t.C) dst[(long long)c * t.d_c + (long long)r * t.d_r] = tile[threadIdx.x][k];
  }
}

// product tables (compile-time): A plane, B plane, accumulator (0 = Re, 1 = Im),
// negate-A flag, and whether the product is the first into its accumulator
template <int NPROD>
struct Prod;
template <>
struct Prod<12> {  // split forms: planes re_hi, re_lo, im_hi, im_lo; hi.hi + hi.lo + lo.hi
  // products 0-5 accumulate Re (Ar.Br terms, then -Ai.Bi terms), 6-11 Im (Ar.Bi, then Ai.Br)
  __host__ __device__ static constexpr int a(int p) {
    return (p % 6) < 2 ? 0 : (p % 6) == 2 ? 1 : (p % 6) < 5 ? 2 : 3;  // hi hi lo | hi hi lo
  }
  __host__ __device__ static constexpr int b(int p) {
    return p < 3 ? (p == 1 ? 1 : 0) : p < 6 ? (p == 4 ? 3 : 2) : p < 9 ? (p == 7 ? 3 : 2) : (p == 10 ? 1 : 0);
  }
  __host__ __device__ static constexpr int acc(int p) { return p < 6 ? 0 : 1; }
  __host__ __device__ static constexpr bool neg(int p) { return p >= 3 && p < 6; }
  __host__ __device__ static constexpr bool first(int p) { return p == 0 || p == 6; }
};
template <>
struct Prod<4> {  // plain tf32: planes re, im
  __host__ __device__ static constexpr int a(int p) { return p == 1 || p == 3 ? 1 : 0; }
  __host__ __device__ static constexpr int b(int p) { return p == 1 || p == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int acc(int p) { return p < 2 ? 0 : 1; }
  __host__ __device__ static constexpr bool neg(int p) { return p == 1; }
  __host__ __device__ static constexpr bool first(int p) { return p == 0 || p == 2; }
};

template <int KIND, int NPROD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);
  // barriers: full[NSTAGE], empty[NSTAGE], tfull[2], tempty[2]; then the TMEM address slot
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSTAGE + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSTAGE);
  const uint32_t tfull0 = smem_u32(bars + 2 * NSTAGE), tempty0 = smem_u32(bars + 2 * NSTAGE + 2);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  const int mt = (a.M + TM - 1) / TM, nt = (a.N + TN - 1) / TN;
  const int ntiles = mt * nt * a.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 4);  // one arrival per epilogue warp
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
  const uint32_t bytesA = a.planes * TM * KCB, bytesB = a.planes * TN * KCB;

  // tile t -> (split z, row tile y, column tile x) and its K-tile range
  // the shorter tile dimension runs fastest, so CTAs that run together share
  // the tiles of the longer operand (read once from DRAM, then from L2)
  auto tile_of = [&](int t, int& m0, int& n0, int& kt0, int& kt1) {
    const int z = t / (mt * nt), r = t % (mt * nt);
    m0 = (mt <= nt ? r % mt : r / nt) * TM;
    n0 = (mt <= nt ? r / mt : r % nt) * TN;
    kt0 = z * a.tiles_per_split;
    kt1 = min(a.k_tiles, kt0 + a.tiles_per_split);
    if (kt1 < kt0) kt1 = kt0;
    return z;
  };

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      const int kc_elems = KCB / a.elem_bytes;
      long long g = 0;  // stage ring counter across tiles
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0, kt0, kt1;
        tile_of(t, m0, n0, kt0, kt1);
        for (int kt = kt0; kt < kt1; ++kt, ++g) {
          const int s = int(g % NSTAGE);
          const uint32_t ph = uint32_t(g / NSTAGE) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err, 1)) {
            ok = false;
            break;
          }
          const uint32_t fb = full0 + 8 * s;
          mbar_expect_tx(fb, bytesA + bytesB);
          const int ko = kt / a.k_in_chunks, kc = (kt % a.k_in_chunks) * kc_elems;
          uint8_t* st = smem + s * STAGE_BYTES;
          tma_load_4d(smem_u32(st), &tmA, kc, ko, m0, 0, fb);
          tma_load_4d(smem_u32(st + A_BYTES), &tmB, kc, ko, n0, 0, fb);
        }
      }
      // do not leave while copies are in flight: wait for the last stages filled
      for (long long q = (g > NSTAGE ? g - NSTAGE : 0); q < g; ++q)
        mbar_wait(full0 + 8 * int(q % NSTAGE), uint32_t(q / NSTAGE) & 1u, a.err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // instruction descriptor: fp32 accumulate, K-major A and B, M = TM, N = TN
      const uint32_t fmtAB = (KIND == TC_BF16) ? 1u : 2u;
      const uint32_t base_id = (1u << 4) | (fmtAB << 7) | (fmtAB << 10) | ((uint32_t)(TN >> 3) << 17) |
                               ((uint32_t)(TM >> 4) << 24);
      long long g = 0;
      int i = 0;  // local tile count
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        int m0, n0, kt0, kt1;
        tile_of(t, m0, n0, kt0, kt1);
        const int b = i & 1;
        // the epilogue must have drained this accumulator buffer (first use passes)
        if (!mbar_wait(tempty0 + 8 * b, (uint32_t(i >> 1) & 1u) ^ 1u, a.err, 5)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)(b * 2 * TN);
        for (int kt = kt0; kt < kt1; ++kt, ++g) {
          const int s = int(g % NSTAGE);
          const uint32_t ph = uint32_t(g / NSTAGE) & 1u;
          if (!mbar_wait(full0 + 8 * s, ph, a.err, 3)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
          // descriptors of plane 0 of this stage; planes and K-steps are fixed offsets
          const uint64_t ad0 = sdesc(sa), bd0 = sdesc(sb);
#pragma unroll
          for (int ks = 0; ks < KCB / 32; ++ks) {
#pragma unroll
            for (int p = 0; p < NPROD; ++p) {
              const uint64_t ad = ad0 + (uint64_t)((Prod<NPROD>::a(p) * TM * KCB + ks * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((Prod<NPROD>::b(p) * TN * KCB + ks * 32) >> 4);
              const uint32_t id = base_id | (Prod<NPROD>::neg(p) ? (1u << 13) : 0u);
              const bool first = (kt == kt0) && ks == 0 && Prod<NPROD>::first(p);
              mma<KIND>(dbase + Prod<NPROD>::acc(p) * TN, ad, bd, id, first ? 0u : 1u);
            }
          }
          mma_commit(empty0 + 8 * s);
        }
        mma_commit(tfull0 + 8 * b);
      }
    }
  } else {
    // epilogue: warps 2..5 own tensor-memory lane quarters (warp % 4)
    const int q = warp % 4;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      int m0, n0, kt0, kt1;
      const int z = tile_of(t, m0, n0, kt0, kt1);
      const bool has_k = kt1 > kt0;
      const int b = i & 1;
      if (!mbar_wait(tfull0 + 8 * b, uint32_t(i >> 1) & 1u, a.err, 4)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m = m0 + q * 32 + lane;
      const uint32_t trow = tmem + (uint32_t)(b * 2 * TN) + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < TN; c0 += 32) {
        uint32_t rr[32], ri[32];
        if (has_k) {
          tmem_ld32(trow + c0, rr);
          tmem_ld32(trow + TN + c0, ri);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) rr[j] = ri[j] = 0u;
        }
        if (m >= a.M) continue;
        const int nb = n0 + c0;
        if (a.out_mode == TC_OUT_PARTIAL) {
          float2* P = a.partial + ((long long)z * a.M + m) * (long long)a.N;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = nb + j;
            if (n < a.N) P[n] = make_float2(__uint_as_float(rr[j]), __uint_as_float(ri[j]));
          }
        } else {
          for (int o = 0; o < a.nout; ++o) {
            const TcOutMap& om = a.out[o];
            const long long mo = (long long)(m / om.M2) * om.sM1 + (long long)(m % om.M2) * om.sM2;
            int n1 = nb / om.N2, n2 = nb % om.N2;
            const long long off0 = mo + (long long)n1 * om.sN1 + n2;
            const int vec = (a.fmt == TC_BF16) ? 8 : 4;  // elements per 16-byte store
            if (om.sN2 == 1 && n2 + 32 <= om.N2 && nb + 32 <= a.N && (off0 % vec) == 0) {
              put_row32(om, a.fmt, off0, rr, ri);
            } else {
              for (int j = 0; j < 32; ++j) {
                if (nb + j < a.N)
                  put(om, a.fmt, mo + (long long)n1 * om.sN1 + (long long)n2 * om.sN2, __uint_as_float(rr[j]),
                      __uint_as_float(ri[j]));
                if (++n2 == om.N2) {
                  n2 = 0;
                  ++n1;
                }
              }
            }
          }
        }
      }
      // this warp is done reading the buffer: hand it back to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * b) : "memory");
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

// fp64 (or fp32 partial) source -> planes, with two-level index maps
__global__ void to_planes_kernel(TcConvert c) {
  const long long total = (long long)c.rows * c.K;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = int(idx / c.K), k = int(idx % c.K);
    const long long so = (long long)(r / c.R2) * c.sR1 + (long long)(r % c.R2) * c.sR2 +
                         (long long)(k / c.K2) * c.sK1 + (long long)(k % c.K2) * c.sK2;
    double2 v = reinterpret_cast<const double2*>(c.src)[so];
    if (c.conj) v.y = -v.y;
    const long long doff = (long long)r * c.row_pitch + (long long)(k / c.kin) * c.kout_pitch + (k % c.kin);
    put(c.dst, c.fmt, doff, float(v.x), float(v.y));
  }
}

// sum split-K partials (fixed order) into fp64 with a strided store
__global__ void reduce_partials_kernel(const float2* P, int splits, int M, int N, double2* out, long long sm,
                                       long long sn) {
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = int(idx / N), n = int(idx % N);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
      float2 v = P[((long long)s * M + m) * N + n];
      re += v.x;
      im += v.y;
    }
    out[m * sm + n * sn] = make_double2(re, im);
  }
}

__global__ void fill_planes_kernel(TcOutMap o, int fmt, long long n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    put(o, fmt, idx, 0.f, 0.f);
}

int grid_for(long long n, int sms) {
  long long b = (n + 255) / 256;
  if (b > 16LL * sms) b = 16LL * sms;
  return int(b < 1 ? 1 : b);
}

}  // namespace

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  // looked up once (a function-local static is initialised once, thread-safely)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

int tc_make_map(CUtensorMap* m, const TcOperand& o, int tile_rows, int box_planes) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return TEVO_ECUDA;
  const int eb = o.elem_bytes;
  if ((reinterpret_cast<uintptr_t>(o.base) & 15) || ((o.row_pitch * eb) & 15) || ((o.kout_pitch * eb) & 15) ||
      ((o.plane_stride * eb) & 15))
    return TEVO_ESHAPE;
  cuuint64_t dims[4] = {(cuuint64_t)o.k_in, (cuuint64_t)o.k_out, (cuuint64_t)o.rows, (cuuint64_t)o.planes};
  cuuint64_t strides[3] = {(cuuint64_t)(o.k_out > 1 ? o.kout_pitch : o.row_pitch) * eb,
                           (cuuint64_t)o.row_pitch * eb, (cuuint64_t)o.plane_stride * eb};
  cuuint32_t box[4] = {(cuuint32_t)(KCB / eb), 1u, (cuuint32_t)tile_rows, (cuuint32_t)box_planes};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, eb == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                   const_cast<void*>(o.base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : TEVO_ESHAPE;
}

int tc_planes(int fmt) { return fmt == TC_TF32 ? 2 : 4; }
int tc_elem_bytes(int fmt) { return fmt == TC_BF16 ? 2 : 4; }
int tc_kchunk(int fmt) { return KCB / tc_elem_bytes(fmt); }

void tc_products(int fmt, TcArgs& a) {
  if (fmt == TC_TF32) {
    // planes: 0 re, 1 im
    const int8_t ap[4] = {0, 1, 0, 1}, bp[4] = {0, 1, 1, 0}, ac[4] = {0, 0, 1, 1}, ng[4] = {0, 1, 0, 0};
    a.nprod = 4;
    for (int i = 0; i < 4; ++i) {
      a.a_plane[i] = ap[i];
      a.b_plane[i] = bp[i];
      a.acc[i] = ac[i];
      a.neg[i] = ng[i];
    }
  } else {
    // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo; hi.hi + hi.lo + lo.hi per real product
    const int8_t ap[12] = {0, 0, 1, 2, 2, 3, 0, 0, 1, 2, 2, 3};
    const int8_t bp[12] = {0, 1, 0, 2, 3, 2, 2, 3, 2, 0, 1, 0};
    const int8_t ac[12] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1};
    const int8_t ng[12] = {0, 0, 0, 1, 1, 1, 0, 0, 0, 0, 0, 0};
    a.nprod = 12;
    for (int i = 0; i < 12; ++i) {
      a.a_plane[i] = ap[i];
      a.b_plane[i] = bp[i];
      a.acc[i] = ac[i];
      a.neg[i] = ng[i];
    }
  }
}

int tc_gemm(const Launch& L, int fmt, const TcOperand& A, const TcOperand& B, int M, int N, TcArgs args) {
  static std::atomic<unsigned long long> attr_done[3];
  const int kind = fmt == TC_BF16 ? 0 : (fmt == TC_TF32X3 ? 1 : 2);
  const int ae = kind == 0   ? smem_attr_once(tc_gemm_kernel<TC_BF16, 12>, SMEM_BYTES, attr_done[0])
                 : kind == 1 ? smem_attr_once(tc_gemm_kernel<TC_TF32, 12>, SMEM_BYTES, attr_done[1])
                             : smem_attr_once(tc_gemm_kernel<TC_TF32, 4>, SMEM_BYTES, attr_done[2]);
  if (ae) return TEVO_ECUDA;
  if (A.k_in != B.k_in || A.k_out != B.k_out || A.planes != B.planes || A.elem_bytes != B.elem_bytes)
    return TEVO_ESHAPE;
  if (A.rows < M || B.rows < N) return TEVO_ESHAPE;
  CUtensorMap ma, mb;
  int e = tc_make_map(&ma, A, TM, A.planes);
  if (!e) e = tc_make_map(&mb, B, TN, B.planes);
  if (e) return e;
  args.M = M;
  args.N = N;
  args.planes = A.planes;
  args.elem_bytes = A.elem_bytes;
  args.fmt = fmt;
  const int kc = KCB / A.elem_bytes;
  args.k_in_chunks = (A.k_in + kc - 1) / kc;
  args.k_tiles = args.k_in_chunks * A.k_out;
  int splits = args.splits < 1 ? 1 : args.splits;
  if (args.out_mode != TC_OUT_PARTIAL) splits = 1;
  args.tiles_per_split = (args.k_tiles + splits - 1) / splits;
  splits = (args.k_tiles + args.tiles_per_split - 1) / args.tiles_per_split;
  args.splits = splits;
  tc_products(fmt, args);
  const long long ntiles = (long long)((N + TN - 1) / TN) * ((M + TM - 1) / TM) * splits;
  if (ntiles > (1LL << 30)) return TEVO_ESHAPE;
  // persistent: one CTA per SM (shared memory allows no more), static tile loop
  dim3 grid((unsigned)std::min<long long>(ntiles, (long long)L.num_sms));
  const double useful = 8.0 * (double)M * N * (double)A.k_in * A.k_out;
  int pr = L.prof ? L.prof->begin(L.stream, TEVO_PROF_GEMMTC, useful,
                                  (double)A.elem_bytes * A.planes * ((double)M + N) * A.k_in * A.k_out)
                  : -1;
  if (kind == 0)
    tc_gemm_kernel<TC_BF16, 12><<<grid, TC_THREADS, SMEM_BYTES, L.stream>>>(ma, mb, args);
  else if (kind == 1)
    tc_gemm_kernel<TC_TF32, 12><<<grid, TC_THREADS, SMEM_BYTES, L.stream>>>(ma, mb, args);
  else
    tc_gemm_kernel<TC_TF32, 4><<<grid, TC_THREADS, SMEM_BYTES, L.stream>>>(ma, mb, args);
  ++*L.launches;
  if (L.prof) L.prof->end(L.stream, pr);
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int tc_to_planes(const Launch& L, const TcConvert& c) {
  const long long total = (long long)c.rows * c.K;
  if (total <= 0) return 0;
  to_planes_kernel<<<grid_for(total, L.num_sms), 256, 0, L.stream>>>(c);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int tc_reduce_partials(const Launch& L, const float2* P, int splits, int M, int N, void* out, long long sm,
                       long long sn) {
  const long long total = (long long)M * N;
  reduce_partials_kernel<<<grid_for(total, L.num_sms), 256, 0, L.stream>>>(P, splits, M, N,
                                                                           reinterpret_cast<double2*>(out), sm, sn);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int tc_transpose(const Launch& L, int fmt, const TcTranspose& t) {
  if (t.R <= 0 || t.C <= 0 || t.batch <= 0) return 0;
  const long long z = (long long)t.batch * tc_planes(fmt);
  if (z > 65535 || (t.R + 31) / 32 > 65535) return TEVO_ESHAPE;
  dim3 grid((t.C + 31) / 32, (t.R + 31) / 32, (unsigned)z), block(32, 8);
  if (fmt == TC_BF16)
    transpose_planes_kernel<unsigned short><<<grid, block, 0, L.stream>>>(t);
  else
    transpose_planes_kernel<unsigned int><<<grid, block, 0, L.stream>>>(t);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int tc_wait_selftest(const Launch& L, int* err_dev, double limit_ms) {
  wait_selftest_kernel<<<1, 32, 0, L.stream>>>(err_dev, (unsigned long long)(limit_ms * 1e6));
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

int tc_zero_planes(const Launch& L, const TcOutMap& o, int fmt, long long n) {
  if (n <= 0) return 0;
  fill_planes_kernel<<<grid_for(n, L.num_sms), 256, 0, L.stream>>>(o, fmt, n);
  ++*L.launches;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

}  // namespace tevo
