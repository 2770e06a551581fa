// Low-precision sweep of evolve_step: the environment and apply contractions
// (G1, G2, G3, G3') on the tensor cores (k_tc.cu), the QR and the site tensors
// in fp64. Operands live between kernels in the plane format of the chosen
// precision; the epilogue of each GEMM writes the next GEMM's operand layout:
//
//   env slot b   [P][D_phi][w][psi_pad]        (view 1: rows (phi w), K = psi;
//                                                view 2: rows phi, K = (w, psi))
//   X^T          [P][(p b)][pad(wl d)]          G1 -> G2 (B operand)
//   T1           [P][(p s)][wr][pad(Db)]        G2 -> G3 (A operand)
//   T2           [P][(v b)][pad(Dp d)]          G2 -> G3' (B operand)
//   site^T       [P][(s' b)][pad(Da)]           fp64 site -> G1 (B operand)
//   Q^H          [P][q][pad(Dp d)]              fp64 QR -> G3' (A operand)
// (P planes, pad = multiple of 8 elements; padded entries are never read: the
// TMA bounds stop at the valid extents).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tevo_mixed.h"
#include "tevo_tc.h"

namespace tevo {

namespace {

#define TRY(x)         \
  do {                 \
    int _e = (x);      \
    if (_e) return _e; \
  } while (0)

inline long long pad8(long long x) { return (x + 7) / 8 * 8; }
inline size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }

int fmt_of(int precision) {
  switch (precision) {
    case TEVO_TF32: return TC_TF32;
    case TEVO_TF32X3: return TC_TF32X3;
    default: return TC_BF16;
  }
}

struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
};

int grow(tevo_ctx c, DevMem& m, size_t bytes) {
  if (m.p && m.bytes >= bytes) return 0;
  ++g_persist_gen;
  if (m.p) ctx_free(c, m.p);
  m.p = nullptr;
  m.bytes = 0;
  TRY(ctx_alloc(c, &m.p, bytes));
  m.bytes = bytes;
  return 0;
}

}  // namespace

struct MixedMPO {
  int fmt = -1;
  std::vector<DevMem> Wr, Wl;  // plane operands of G2
};

struct MixedState {
  int fmt = -1;
  std::vector<size_t> env_off;
  std::vector<int> env_w;
  DevMem env, Xn, Xt, T1, T2, site, Qp, part, err;
};

namespace {

int P_(int fmt) { return tc_planes(fmt); }
int EB(int fmt) { return tc_elem_bytes(fmt); }

struct Dims {
  int Dp, Da, wl, d, Db, Dq, wr;
};

char* envp(MixedState* m, int b) { return static_cast<char*>(m->env.p) + m->env_off[b]; }

long long env_plane_stride(const std::vector<int>& dims, int w, int b) {
  return (long long)dims[b] * w * pad8(dims[b]);
}

// view 1 of an environment: rows (phi w), K = psi
TcOperand env_view1(MixedState* m, const std::vector<int>& dims, int b, int fmt) {
  const int w = m->env_w[b];
  TcOperand o;
  o.base = envp(m, b);
  o.elem_bytes = EB(fmt);
  o.planes = P_(fmt);
  o.plane_stride = env_plane_stride(dims, w, b);
  o.rows = dims[b] * w;
  o.row_pitch = pad8(dims[b]);
  o.k_in = dims[b];
  o.k_out = 1;
  o.kout_pitch = o.row_pitch;
  return o;
}

// view 2 of an environment: rows phi, K = (w, psi)
TcOperand env_view2(MixedState* m, const std::vector<int>& dims, int b, int fmt) {
  const int w = m->env_w[b];
  TcOperand o;
  o.base = envp(m, b);
  o.elem_bytes = EB(fmt);
  o.planes = P_(fmt);
  o.plane_stride = env_plane_stride(dims, w, b);
  o.rows = dims[b];
  o.row_pitch = (long long)w * pad8(dims[b]);
  o.k_in = dims[b];
  o.k_out = w;
  o.kout_pitch = pad8(dims[b]);
  return o;
}

TcOutMap env_out(MixedState* m, const std::vector<int>& dims, int b) {
  const int w = m->env_w[b];
  const long long bp = pad8(dims[b]);
  TcOutMap o;
  o.base = envp(m, b);
  o.plane_stride = env_plane_stride(dims, w, b);
  o.M2 = 1 << 30;
  o.sM1 = 0;
  o.sM2 = (long long)w * bp;
  o.N2 = dims[b];
  o.sN1 = bp;
  o.sN2 = 1;
  return o;
}

TcArgs base_args(MixedState* m) {
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.err = static_cast<int*>(m->err.p);
  a.splits = 1;
  a.out_mode = TC_OUT_PLANES;
  return a;
}

// plane operand of a site tensor read as G1's B: rows (s' b), K = a.
// mirrored = false: A[a][s'][b] = site[a][s'][b]        (site [Da][d][Db])
// mirrored = true : A[a][s'][b] = site[b][s'][a]        (site [Db][d][Da])
int convert_site(tevo_ctx c, MixedState* m, const void* site, const Dims& k, bool mirrored, int fmt) {
  TcConvert cv;
  std::memset(&cv, 0, sizeof(cv));
  cv.src = site;
  cv.rows = k.d * k.Db;
  cv.K = k.Da;
  if (!mirrored) {
    cv.R2 = cv.rows;
    cv.sR1 = 0;
    cv.sR2 = 1;
    cv.K2 = cv.K;
    cv.sK1 = 0;
    cv.sK2 = (long long)k.d * k.Db;
  } else {
    cv.R2 = k.Db;                 // n = s' * Db + b
    cv.sR1 = k.Da;                // s'
    cv.sR2 = (long long)k.d * k.Da;  // b
    cv.K2 = cv.K;
    cv.sK1 = 0;
    cv.sK2 = 1;
  }
  cv.conj = 0;
  cv.fmt = fmt;
  cv.dst.base = m->site.p;
  cv.dst.plane_stride = (long long)cv.rows * pad8(k.Da);
  cv.row_pitch = pad8(k.Da);
  cv.kin = cv.K;
  cv.kout_pitch = 0;
  return tc_to_planes(ctx_launch(c), cv);
}

TcOperand site_operand(MixedState* m, const Dims& k, int fmt) {
  TcOperand o;
  o.base = m->site.p;
  o.elem_bytes = EB(fmt);
  o.planes = P_(fmt);
  o.rows = k.d * k.Db;
  o.row_pitch = pad8(k.Da);
  o.plane_stride = (long long)o.rows * o.row_pitch;
  o.k_in = k.Da;
  o.k_out = 1;
  o.kout_pitch = o.row_pitch;
  return o;
}

// conj of a matrix read as G3''s A: rows q (Dq), K = (p s) (Dp d).
// from_colmajor: Q column-major (m = Dp d rows, Dq cols): A(q, k) = conj(Q[k + q * m])
// otherwise from a site tensor in the mirrored layout: A(l, (r s)) = conj(site[l][s][r]),
// site [Dq][d][Dp] (the bra of an environment build)
int convert_q(tevo_ctx c, MixedState* m, const void* src, const Dims& k, bool from_colmajor, int fmt) {
  TcConvert cv;
  std::memset(&cv, 0, sizeof(cv));
  cv.src = src;
  cv.rows = k.Dq;
  cv.K = k.Dp * k.d;
  cv.R2 = cv.rows;
  cv.sR1 = 0;
  if (from_colmajor) {
    cv.sR2 = (long long)k.Dp * k.d;
    cv.K2 = cv.K;
    cv.sK1 = 0;
    cv.sK2 = 1;
  } else {
    cv.sR2 = (long long)k.d * k.Dp;  // l
    cv.K2 = k.d;                     // k = r * d + s
    cv.sK1 = 1;                      // r
    cv.sK2 = k.Dp;                   // s
  }
  cv.conj = 1;
  cv.fmt = fmt;
  cv.dst.base = m->Qp.p;
  cv.dst.plane_stride = (long long)cv.rows * pad8(cv.K);
  cv.row_pitch = pad8(cv.K);
  cv.kin = cv.K;
  cv.kout_pitch = 0;
  return tc_to_planes(ctx_launch(c), cv);
}

TcOperand q_operand(MixedState* m, const Dims& k, int fmt) {
  TcOperand o;
  o.base = m->Qp.p;
  o.elem_bytes = EB(fmt);
  o.planes = P_(fmt);
  o.rows = k.Dq;
  o.row_pitch = pad8((long long)k.Dp * k.d);
  o.plane_stride = (long long)o.rows * o.row_pitch;
  o.k_in = k.Dp * k.d;
  o.k_out = 1;
  o.kout_pitch = o.row_pitch;
  return o;
}

TcOperand w_operand(const DevMem& w, const Dims& k, int fmt) {
  TcOperand o;
  o.base = w.p;
  o.elem_bytes = EB(fmt);
  o.planes = P_(fmt);
  o.rows = k.d * k.wr;
  o.row_pitch = pad8((long long)k.wl * k.d);
  o.plane_stride = (long long)o.rows * o.row_pitch;
  o.k_in = k.wl * k.d;
  o.k_out = 1;
  o.kout_pitch = o.row_pitch;
  return o;
}

// G1 + G2: T1 and T2 from (env view 1 of slot_left, site planes, W planes).
// G1 writes X row-contiguous ([(p w)][(s' b)]); a batched transpose gives the
// K-major X^T[(p b)][(w s')] that G2 reads; G2 writes T1 row-contiguous and a
// second transpose gives T2 = T1^T for G3'.
int make_T(tevo_ctx c, MixedState* m, const std::vector<int>& dims, int slot_left, const DevMem& Wp, const Dims& k,
           int fmt, bool want_T1) {
  (void)want_T1;
  const Launch L = ctx_launch(c);
  const int P = P_(fmt);
  const long long npad = pad8((long long)k.d * k.Db);
  const long long kp2 = pad8((long long)k.wl * k.d);
  const long long bp = pad8(k.Db), kp4 = pad8((long long)k.Dp * k.d);
  // G1: X(m = (p w), n = (s' b)) -> X[(p w)][(s' b)]
  {
    TcArgs a = base_args(m);
    a.nout = 1;
    a.out[0].base = m->Xn.p;
    a.out[0].plane_stride = (long long)k.Dp * k.wl * npad;
    a.out[0].M2 = 1 << 30;
    a.out[0].sM1 = 0;
    a.out[0].sM2 = npad;
    a.out[0].N2 = 1 << 30;
    a.out[0].sN1 = 0;
    a.out[0].sN2 = 1;
    TRY(tc_gemm(L, fmt, env_view1(m, dims, slot_left, fmt), site_operand(m, k, fmt), k.Dp * k.wl, k.d * k.Db, a));
  }
  // X^T[(p b)][(w s')]: per (p, s'), transpose the wl x Db block
  {
    TcTranspose t;
    t.src = m->Xn.p;
    t.dst = m->Xt.p;
    t.src_plane = (long long)k.Dp * k.wl * npad;
    t.dst_plane = (long long)k.Dp * k.Db * kp2;
    t.batch = k.Dp * k.d;
    t.B2 = k.d;
    t.sb1 = (long long)k.wl * npad;
    t.sb2 = k.Db;
    t.db1 = (long long)k.Db * kp2;
    t.db2 = 1;
    t.R = k.wl;
    t.C = k.Db;
    t.s_r = npad;
    t.d_c = kp2;
    t.d_r = k.d;
    TRY(tc_transpose(L, fmt, t));
  }
  // G2: T(m = (s v), n = (p b)) -> T1[(p s)][v][b]
  {
    TcOperand B;
    B.base = m->Xt.p;
    B.elem_bytes = EB(fmt);
    B.planes = P;
    B.rows = k.Dp * k.Db;
    B.row_pitch = kp2;
    B.plane_stride = (long long)B.rows * kp2;
    B.k_in = k.wl * k.d;
    B.k_out = 1;
    B.kout_pitch = kp2;
    TcArgs a = base_args(m);
    TcOutMap& o = a.out[0];
    o.base = m->T1.p;
    o.plane_stride = (long long)k.Dp * k.d * k.wr * bp;
    o.M2 = k.wr;
    o.sM1 = (long long)k.wr * bp;
    o.sM2 = bp;
    o.N2 = k.Db;
    o.sN1 = (long long)k.d * k.wr * bp;
    o.sN2 = 1;
    a.nout = 1;
    TRY(tc_gemm(L, fmt, w_operand(Wp, k, fmt), B, k.d * k.wr, k.Dp * k.Db, a));
  }
  // T2[(v b)][(p s)] = T1^T, batched over v
  {
    TcTranspose t;
    t.src = m->T1.p;
    t.dst = m->T2.p;
    t.src_plane = (long long)k.Dp * k.d * k.wr * bp;
    t.dst_plane = (long long)k.wr * k.Db * kp4;
    t.batch = k.wr;
    t.B2 = k.wr;
    t.sb1 = 0;
    t.sb2 = bp;
    t.db1 = 0;
    t.db2 = (long long)k.Db * kp4;
    t.R = k.Dp * k.d;
    t.C = k.Db;
    t.s_r = (long long)k.wr * bp;
    t.d_c = kp4;
    t.d_r = 1;
    TRY(tc_transpose(L, fmt, t));
  }
  return 0;
}

// G3: B = T1 . Er^T into the fp64 column-major buffer of the QR
int apply_tc(tevo_ctx c, MixedState* m, const std::vector<int>& dims, int slot_right, const Dims& k, int fmt,
             void* Bq, int num_sms) {
  const Launch L = ctx_launch(c);
  const long long bp = pad8(k.Db);
  TcOperand A;
  A.base = m->T1.p;
  A.elem_bytes = EB(fmt);
  A.planes = P_(fmt);
  A.rows = k.Dp * k.d;
  A.row_pitch = (long long)k.wr * bp;
  A.plane_stride = (long long)A.rows * A.row_pitch;
  A.k_in = k.Db;
  A.k_out = k.wr;
  A.kout_pitch = bp;
  const int M = k.Dp * k.d, N = k.Dq;
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
  const int kc = tc_kchunk(fmt);
  const int ktiles = ((k.Db + kc - 1) / kc) * k.wr;
  int splits = std::max(1, std::min(num_sms / std::max(1, tiles), ktiles / 2));
  splits = std::min(splits, 64);
  TcArgs a = base_args(m);
  a.out_mode = TC_OUT_PARTIAL;
  a.splits = splits;
  a.partial = static_cast<float2*>(m->part.p);
  // the engine may lower the split count so that no split is empty
  const int tps = (ktiles + splits - 1) / splits;
  const int used = (ktiles + tps - 1) / tps;
  TRY(tc_gemm(L, fmt, A, env_view2(m, dims, slot_right, fmt), M, N, a));
  return tc_reduce_partials(L, static_cast<float2*>(m->part.p), used, M, N, Bq, 1, M);
}

// G3': new environment (slot_out) from the Q^H planes and T2
int env_tc(tevo_ctx c, MixedState* m, const std::vector<int>& dims, int slot_out, const Dims& k, int fmt) {
  const Launch L = ctx_launch(c);
  const long long kp4 = pad8((long long)k.Dp * k.d);
  TcOperand B;
  B.base = m->T2.p;
  B.elem_bytes = EB(fmt);
  B.planes = P_(fmt);
  B.rows = k.wr * k.Db;
  B.row_pitch = kp4;
  B.plane_stride = (long long)B.rows * kp4;
  B.k_in = k.Dp * k.d;
  B.k_out = 1;
  B.kout_pitch = kp4;
  TcArgs a = base_args(m);
  a.nout = 1;
  a.out[0] = env_out(m, dims, slot_out);
  return tc_gemm(L, fmt, q_operand(m, k, fmt), B, k.Dq, k.wr * k.Db, a);
}

Dims right_dims(tevo_mpo W, const std::vector<int>& dims, int d, int i) {
  return Dims{dims[i], dims[i], mpo_wl(W, i), d, dims[i + 1], dims[i + 1], mpo_wr(W, i)};
}
Dims left_dims(tevo_mpo W, const std::vector<int>& dims, int d, int i) {
  return Dims{dims[i + 1], dims[i + 1], mpo_wr(W, i), d, dims[i], dims[i], mpo_wl(W, i)};
}

int set_boundary_env(tevo_ctx c, tevo_mps s, MixedState* m, int b, int fmt) {
  const std::vector<int>& dims = mps_dims(s);
  TcConvert cv;
  std::memset(&cv, 0, sizeof(cv));
  cv.src = mps_env_slot(s, b);  // fp64 slot holds the scalar 1
  cv.rows = 1;
  cv.K = 1;
  cv.R2 = 1;
  cv.K2 = 1;
  cv.fmt = fmt;
  cv.dst.base = envp(m, b);
  cv.dst.plane_stride = env_plane_stride(dims, m->env_w[b], b);
  cv.row_pitch = 8;
  cv.kin = 1;
  return tc_to_planes(ctx_launch(c), cv);
}

}  // namespace

int mixed_prepare(tevo_ctx c, tevo_mpo W, tevo_mps s, int precision) {
  const int fmt = fmt_of(precision);
  const int L = mps_L(s), d = mps_d(s);
  const std::vector<int>& dims = mps_dims(s);
  const int P = P_(fmt), eb = EB(fmt);
  MixedMPO*& mm = mpo_mixed(W);
  if (!mm) mm = new MixedMPO;
  if (mm->fmt != fmt) {
    ++g_persist_gen;
    mm->Wr.resize(L);
    mm->Wl.resize(L);
    for (int i = 0; i < L; ++i) {
      const int wl = mpo_wl(W, i), wr = mpo_wr(W, i);
      for (int side = 0; side < 2; ++side) {
        const int rows = d * (side == 0 ? wr : wl), K = d * (side == 0 ? wl : wr);
        DevMem& dm = side == 0 ? mm->Wr[i] : mm->Wl[i];
        TRY(grow(c, dm, al((size_t)P * rows * pad8(K) * eb)));
        TcConvert cv;
        std::memset(&cv, 0, sizeof(cv));
        cv.src = side == 0 ? mpo_dev_wr(W, i) : mpo_dev_wl(W, i);
        cv.rows = rows;
        cv.K = K;
        cv.R2 = rows;
        cv.sR2 = K;
        cv.K2 = K;
        cv.sK2 = 1;
        cv.fmt = fmt;
        cv.dst.base = dm.p;
        cv.dst.plane_stride = (long long)rows * pad8(K);
        cv.row_pitch = pad8(K);
        cv.kin = K;
        TRY(tc_to_planes(ctx_launch(c), cv));
      }
    }
    mm->fmt = fmt;
  }
  MixedState*& ms = mps_mixed(s);
  if (!ms) ms = new MixedState;
  MixedState* m = ms;
  m->fmt = fmt;
  m->env_off.assign(L + 1, 0);
  m->env_w.assign(L + 1, 1);
  size_t off = 0;
  for (int b = 0; b <= L; ++b) {
    m->env_w[b] = (b == 0 || b == L) ? 1 : mpo_wr(W, b - 1);
    m->env_off[b] = off;
    off += al((size_t)P * env_plane_stride(dims, m->env_w[b], b) * eb);
  }
  TRY(grow(c, m->env, off));
  size_t xn = 0, xt = 0, t1 = 0, t2 = 0, site = 0, qp = 0, part = 0;
  for (int i = 0; i < L; ++i) {
    for (int side = 0; side < 2; ++side) {
      Dims k = side == 0 ? right_dims(W, dims, d, i) : left_dims(W, dims, d, i);
      xt = std::max<size_t>(xt, (size_t)P * k.Dp * k.Db * pad8((long long)k.wl * k.d) * eb);
      xn = std::max<size_t>(xn, (size_t)P * k.Dp * k.wl * pad8((long long)k.d * k.Db) * eb);
      t1 = std::max<size_t>(t1, (size_t)P * k.Dp * k.d * k.wr * pad8(k.Db) * eb);
      t2 = std::max<size_t>(t2, (size_t)P * k.wr * k.Db * pad8((long long)k.Dp * k.d) * eb);
      site = std::max<size_t>(site, (size_t)P * k.d * k.Db * pad8(k.Da) * eb);
      qp = std::max<size_t>(qp, (size_t)P * k.Dq * pad8((long long)k.Dp * k.d) * eb);
      part = std::max<size_t>(part, (size_t)64 * k.Dp * k.d * k.Dq * 8);
    }
  }
  TRY(grow(c, m->Xn, al(xn)));
  TRY(grow(c, m->Xt, al(xt)));
  TRY(grow(c, m->T1, al(t1)));
  TRY(grow(c, m->T2, al(t2)));
  TRY(grow(c, m->site, al(site)));
  TRY(grow(c, m->Qp, al(qp)));
  TRY(grow(c, m->part, al(part)));
  TRY(grow(c, m->err, 256));
  if (cudaMemsetAsync(m->err.p, 0, 4, ctx_launch(c).stream) != cudaSuccess) return TEVO_ECUDA;
  return 0;
}

int mixed_build_right_envs(tevo_ctx c, tevo_mpo W, tevo_mps s, bool bra_fresh, int precision) {
  MixedState* m = mps_mixed(s);
  MixedMPO* mm = mpo_mixed(W);
  const int fmt = m->fmt;
  const int L = mps_L(s), d = mps_d(s);
  const std::vector<int>& dims = mps_dims(s);
  TRY(set_boundary_env(c, s, m, 0, fmt));
  TRY(set_boundary_env(c, s, m, L, fmt));
  for (int i = L - 1; i >= 1; --i) {
    Dims k = left_dims(W, dims, d, i);
    TRY(convert_site(c, m, mps_site(s, i, false), k, true, fmt));
    TRY(make_T(c, m, dims, i + 1, mm->Wl[i], k, fmt, false));
    TRY(convert_q(c, m, mps_site(s, i, bra_fresh), k, false, fmt));
    TRY(env_tc(c, m, dims, i, k, fmt));
  }
  return 0;
}

int mixed_sweep(tevo_ctx c, tevo_mpo W, tevo_mps s, int precision) {
  MixedState* m = mps_mixed(s);
  MixedMPO* mm = mpo_mixed(W);
  const int fmt = m->fmt;
  const int L = mps_L(s), d = mps_d(s);
  const std::vector<int>& dims = mps_dims(s);
  const int sms = ctx_launch(c).num_sms;
  for (int i = 0; i + 1 < L; ++i) {
    Dims k = right_dims(W, dims, d, i);
    TRY(convert_site(c, m, mps_site(s, i, false), k, false, fmt));
    TRY(make_T(c, m, dims, i, mm->Wr[i], k, fmt, true));
    TRY(apply_tc(c, m, dims, i + 1, k, fmt, mps_buf_Bq(s), sms));
    TRY(mps_qr_q(s, k.Dp * d, k.Dq));
    TRY(mps_store_right(s, i));
    TRY(convert_q(c, m, mps_buf_Bq(s), k, true, fmt));
    TRY(env_tc(c, m, dims, i + 1, k, fmt));
  }
  for (int i = L - 1; i >= 1; --i) {
    Dims k = left_dims(W, dims, d, i);
    TRY(convert_site(c, m, mps_site(s, i, false), k, true, fmt));
    TRY(make_T(c, m, dims, i + 1, mm->Wl[i], k, fmt, true));
    TRY(apply_tc(c, m, dims, i, k, fmt, mps_buf_Bq(s), sms));
    TRY(mps_qr_q(s, k.Dp * d, k.Dq));
    TRY(mps_store_left(s, i));
    TRY(convert_q(c, m, mps_buf_Bq(s), k, true, fmt));
    TRY(env_tc(c, m, dims, i, k, fmt));
  }
  return 0;
}

int mixed_centre(tevo_ctx c, tevo_mpo W, tevo_mps s, int precision) {
  MixedState* m = mps_mixed(s);
  MixedMPO* mm = mpo_mixed(W);
  const int fmt = m->fmt;
  const int d = mps_d(s);
  const std::vector<int>& dims = mps_dims(s);
  Dims k = left_dims(W, dims, d, 0);
  TRY(convert_site(c, m, mps_site(s, 0, false), k, true, fmt));
  TRY(make_T(c, m, dims, 1, mm->Wl[0], k, fmt, true));
  TRY(apply_tc(c, m, dims, 0, k, fmt, mps_buf_Bq(s), ctx_launch(c).num_sms));
  return mps_store_left(s, 0);
}

int mixed_error_flag(tevo_ctx c, tevo_mps s, int* flag) {
  MixedState* m = mps_mixed(s);
  *flag = 0;
  if (!m || !m->err.p) return 0;
  if (cudaMemcpyAsync(flag, m->err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx_launch(c).stream) != cudaSuccess)
    return TEVO_ECUDA;
  return 0;
}

int mixed_gemm(tevo_ctx c, int precision, int M, int N, int K, const void* A, const void* B, void* C) {
  const int fmt = fmt_of(precision);
  const int P = P_(fmt), eb = EB(fmt);
  const Launch L = ctx_launch(c);
  const long long kp = pad8(K);
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
  const int kc = tc_kchunk(fmt);
  const int ktiles = (K + kc - 1) / kc;
  int splits = std::max(1, std::min({L.num_sms / std::max(1, tiles), ktiles, 64}));
  DevMem pa, pb, part, err;
  auto release = [&]() {
    for (DevMem* d : {&pa, &pb, &part, &err})
      if (d->p) ctx_free(c, d->p);
  };
  auto run = [&]() -> int {
    TRY(grow(c, pa, al((size_t)P * M * kp * eb)));
    TRY(grow(c, pb, al((size_t)P * N * kp * eb)));
    TRY(grow(c, part, al((size_t)splits * M * N * 8)));
    TRY(grow(c, err, 256));
    if (cudaMemsetAsync(err.p, 0, 4, L.stream) != cudaSuccess) return TEVO_ECUDA;
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
      cv.dst.base = side == 0 ? pa.p : pb.p;
      cv.dst.plane_stride = (long long)cv.rows * kp;
      cv.row_pitch = kp;
      cv.kin = K;
      TRY(tc_to_planes(L, cv));
    }
    TcOperand oa{pa.p, eb, P, (long long)M * kp, M, kp, K, 1, kp};
    TcOperand ob{pb.p, eb, P, (long long)N * kp, N, kp, K, 1, kp};
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.err = static_cast<int*>(err.p);
    a.out_mode = TC_OUT_PARTIAL;
    a.splits = splits;
    a.partial = static_cast<float2*>(part.p);
    const int tps = (ktiles + splits - 1) / splits;
    const int used = (ktiles + tps - 1) / tps;
    TRY(tc_gemm(L, fmt, oa, ob, M, N, a));
    TRY(tc_reduce_partials(L, static_cast<float2*>(part.p), used, M, N, C, N, 1));
    int flag = 0;
    if (cudaMemcpyAsync(&flag, err.p, sizeof(int), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
        cudaStreamSynchronize(L.stream) != cudaSuccess)
      return TEVO_ECUDA;
    return flag ? TEVO_ETIMEOUT : 0;
  };
  int e = run();
  release();
  return e;
}

void mixed_mpo_destroy(tevo_ctx c, MixedMPO*& m) {
  if (!m) return;
  for (auto& w : m->Wr)
    if (w.p) ctx_free(c, w.p);
  for (auto& w : m->Wl)
    if (w.p) ctx_free(c, w.p);
  delete m;
  m = nullptr;
}

void mixed_state_destroy(tevo_ctx c, MixedState*& m) {
  if (!m) return;
  for (DevMem* d : {&m->env, &m->Xn, &m->Xt, &m->T1, &m->T2, &m->site, &m->Qp, &m->part, &m->err})
    if (d->p) ctx_free(c, d->p);
  delete m;
  m = nullptr;
}

}  // namespace tevo
