// Tensor-core complex GEMM engine (k_tc.cu).
#pragma once

#include <cstdint>

#include "tevo_internal.h"

#ifdef __CUDACC__
#include <vector_types.h>
#else
struct float2 {
  float x, y;
};
#endif

namespace tevo {

// plane formats of the low-precision operands (also the MMA kind)
enum { TC_BF16 = 0, TC_TF32 = 1, TC_TF32X3 = 2 };
enum { TC_OUT_PARTIAL = 0, TC_OUT_PLANES = 1 };

// K-major operand: element (plane p, row r, k = k_out * k_in + k_in_idx) at
// base + p * plane_stride + r * row_pitch + k_out * kout_pitch + k_in_idx (elements).
struct TcOperand {
  const void* base;
  int elem_bytes;
  int planes;
  long long plane_stride;
  int rows;
  long long row_pitch;
  int k_in, k_out;
  long long kout_pitch;
};

// output of the epilogue in plane format: (m, n) goes to
// (m / M2) * sM1 + (m % M2) * sM2 + (n / N2) * sN1 + (n % N2) * sN2 of every plane
struct TcOutMap {
  void* base;
  long long plane_stride;
  int M2;
  long long sM1, sM2;
  int N2;
  long long sN1, sN2;
};

struct TcArgs {
  int M, N;
  int planes, elem_bytes, fmt;
  int k_in_chunks, k_tiles, tiles_per_split, splits;
  int nprod;
  int8_t a_plane[12], b_plane[12], acc[12], neg[12];
  int out_mode;
  int nout;
  TcOutMap out[2];
  float2* partial;  // [splits][M][N] when out_mode == TC_OUT_PARTIAL
  int* err;         // device flag: bounded wait gave up
};

// fp64 complex source -> plane-format operand
struct TcConvert {
  const void* src;  // double2
  int rows, K;
  int R2;
  long long sR1, sR2;
  int K2;
  long long sK1, sK2;
  int conj;
  int fmt;
  TcOutMap dst;     // only base and plane_stride are used
  long long row_pitch, kout_pitch;
  int kin;          // K index k -> (k / kin) * kout_pitch + k % kin
};

// batched plane transpose: for every plane and batch index b (split b = (b / B2, b % B2)),
// dst[c * d_c + r * d_r] = src[r * s_r + c] for r < R, c < C (offsets in elements,
// relative to the batch bases (b / B2) * sb1 + (b % B2) * sb2 and db1, db2)
struct TcTranspose {
  const void* src;
  void* dst;
  long long src_plane, dst_plane;
  int batch, B2;
  long long sb1, sb2, db1, db2;
  int R, C;
  long long s_r, d_c, d_r;
};

int tc_planes(int fmt);
int tc_elem_bytes(int fmt);
int tc_kchunk(int fmt);
int tc_gemm(const Launch& L, int fmt, const TcOperand& A, const TcOperand& B, int M, int N, TcArgs args);
int tc_to_planes(const Launch& L, const TcConvert& c);
int tc_reduce_partials(const Launch& L, const float2* P, int splits, int M, int N, void* out, long long sm,
                       long long sn);
int tc_transpose(const Launch& L, int fmt, const TcTranspose& t);
int tc_wait_selftest(const Launch& L, int* err_dev, double limit_ms);
int tc_zero_planes(const Launch& L, const TcOutMap& o, int fmt, long long n);

}  // namespace tevo
