// C ABI and the host-side sweep driver of libtevo (see include/tevo.h).
//
// Data layout in device memory (complex fp64 as interleaved doubles):
//   MPS site i        A_i[D_i][d][D_{i+1}]          (two sets: psi and the fitted phi)
//   MPO site i        W_i[wl][d][d][wr]             (plus the G2 operands below)
//                     Wr_i[(s wr)][(wl s')]          rightward step
//                     Wl_i[(s wl)][(wr s')]          leftward step (mirrored chain)
//   environment slot b (bond b = 0..L): [D_b][w_b][D_b]; it holds the left
//   environment of <phi|W|psi> for bonds left of the sweep position and the
//   right environment for the others, so one slab of L+1 slots serves both.
//
// A site step in the rightward layout (El, A, W, Er) -> (Q, Enew) is
//   G1  X[(p w), (s' b)]  = El[(p w), a] A[a, (s' b)]
//   G2  T_p[(s v), b]     = Wr[(s v), (w s')] X_p[(w s'), b]        (batched over p)
//   G3  B[(p s), q]       = T[(p s), (v b)] Er[q, (v b)]            (column-major out)
//   QR  B = Q R (Householder, fp64)
//   G3' Enew[q, (v b)]    = conj(Q)[(p s), q] T[(p s), (v b)]
// and the leftward step is the same on the mirrored chain: the site tensor is
// transposed A^T[r][s][l], the environments swap roles and Wl replaces Wr.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tevo_internal.h"
#include "tevo_mixed.h"
#include "tevo_tc.h"

using namespace tevo;

namespace tevo {
long long g_persist_gen = 0;
}

struct tevo_ctx_s {
  cudaStream_t stream = nullptr;
  tevo_alloc_fn alloc = nullptr;
  tevo_free_fn free_fn = nullptr;
  void* user = nullptr;
  long long launches = 0;
  int device = 0;
  int num_sms = 1;
  Prof prof;
};

namespace {

#define TRY(x)                  \
  do {                          \
    int _e = (x);               \
    if (_e) return _e;          \
  } while (0)
#define TRYCUDA(x)                                  \
  do {                                              \
    if ((x) != cudaSuccess) return TEVO_ECUDA;      \
  } while (0)

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

int dalloc(tevo_ctx c, Buf& b, size_t bytes) {
  b.bytes = bytes;
  b.p = nullptr;
  if (bytes == 0) return 0;
  if (c->alloc) {
    b.p = c->alloc(bytes, c->user);
  } else {
    if (cudaMallocAsync(&b.p, bytes, c->stream) != cudaSuccess) b.p = nullptr;
  }
  return b.p ? 0 : TEVO_ENOMEM;
}

void dfree(tevo_ctx c, Buf& b) {
  if (!b.p) return;
  if (c->free_fn)
    c->free_fn(b.p, c->user);
  else
    cudaFreeAsync(b.p, c->stream);
  b.p = nullptr;
  b.bytes = 0;
}

int ensure(tevo_ctx c, Buf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return 0;
  ++g_persist_gen;
  dfree(c, b);
  return dalloc(c, b, bytes);
}

Launch launch_of(tevo_ctx c) { return Launch{c->stream, &c->launches, c->num_sms, &c->prof}; }

inline z64* zp(const Buf& b) { return reinterpret_cast<z64*>(b.p); }

}  // namespace

struct tevo_mpo_s {
  tevo_ctx ctx = nullptr;
  int L = 0, d = 0, chi = 0, N = 0, variant = 0;
  double tau_re = 0, tau_im = 0;
  std::vector<int> wl, wr;
  std::vector<Buf> W, Wr, Wl;
  // nonzeros of Wr / Wl as CSR (row_ptr | col_idx ints, values complex) for G2
  std::vector<Buf> Sr_idx, Sr_val, Sl_idx, Sl_val;
  std::vector<std::vector<std::complex<double>>> host;  // W_i on the host (test access)
  MixedMPO* mixed = nullptr;                            // low-precision operands (lazy)
};

struct tevo_mps_s {
  tevo_ctx ctx = nullptr;
  int L = 0, d = 0, D = 0;
  std::vector<int> dims;
  std::vector<Buf> A, Anew;
  bool canonical = false;
  int parity = 0;  // flips with every psi/phi swap
  Buf scalars;  // [0] lognorm, [1] nrm2, [2] overlap log acc, [3..] flags/values
  // workspace of evolve_step
  std::vector<size_t> env_off;
  Buf env, X, T, Bq, V, tau, beta, Atmp, Rm, gemm_ws, red;
  Buf qrflags;        // [0] error flag of the cooperative QR, [1..] reflector flags
  Buf qrwy;           // Gram matrices and triangular factors of the WY blocks (Q formation)
  Buf T2, Th, jac;    // two-site form: the partner site's T, the two-site matrix, Jacobi workspace
  int qr_epoch = 0;
  bool coop_qr = true;  // off while a batched step issues (concurrent streams, graph capture)
  int oz_slices = 0;    // > 0 while a step runs its fp64 contractions as Ozaki-scheme GEMMs
  bool two_site = false;  // the step in progress fits pairs of sites (TEVO_TWO_SITE)
  Buf oz_ws;            // digit slices, row exponents and split partials of those GEMMs
  int wmax = 0;
  MixedState* mixed = nullptr;
};

namespace {

double* scal(tevo_mps s, int k) { return reinterpret_cast<double*>(s->scalars.p) + k; }

// slot of the scalars buffer holding the device error flag of the Ozaki GEMMs
constexpr int OZ_FLAG_SLOT = 5;

int gemm(tevo_mps s, const GemmDesc& g) {
  Launch L = launch_of(s->ctx);
  if (s->oz_slices > 0) {
    const size_t need = ozgemm64_workspace(g, s->oz_slices, L.num_sms);
    if (need > 0) {
      TRY(ensure(s->ctx, s->oz_ws, need));
      const int e = ozgemm64(L, g, s->oz_slices, s->oz_ws.p, s->oz_ws.bytes,
                             reinterpret_cast<int*>(scal(s, OZ_FLAG_SLOT)));
      if (e != TEVO_EUNSUPPORTED) return e;
    }
  }
  return zgemm64(L, g, s->gemm_ws.p, s->gemm_ws.bytes);
}

GemmDesc gd(const void* A, long long sAb, long long sAm, long long sAk, const void* B, long long sBb,
            long long sBk, long long sBn, void* C, long long sCb, long long sCm, long long sCn, int M,
            int N, int K, int batch, int conjA = 0) {
  GemmDesc g;
  g.A = A;
  g.B = B;
  g.C = C;
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.sAb = sAb;
  g.sAm = sAm;
  g.sAk = sAk;
  g.sBb = sBb;
  g.sBk = sBk;
  g.sBn = sBn;
  g.sCb = sCb;
  g.sCm = sCm;
  g.sCn = sCn;
  g.conjA = conjA;
  g.conjB = 0;
  g.alpha_re = 1;
  g.alpha_im = 0;
  g.beta_re = 0;
  g.beta_im = 0;
  return g;
}

z64* env_slot(tevo_mps s, int b) { return reinterpret_cast<z64*>(static_cast<char*>(s->env.p) + s->env_off[b]); }

// sizes of one site step in the rightward layout
struct StepDims {
  int Dp, Da, wl, d, Db, Dq, wr;
};

// G1 + G2: T from (El, A, Wg) in fp64; G2 skips the MPO's zero entries when
// its CSR form (sidx = row_ptr then col_idx, sval) is given
int make_T64(tevo_mps s, const StepDims& k, const z64* El, const z64* A, const z64* Wg, const Buf* sidx = nullptr,
             const Buf* sval = nullptr, void* Tout = nullptr) {
  void* T = Tout ? Tout : s->T.p;
  // G1: X[(p w), (s' b)] = El[(p w), a] A[a, (s' b)]
  TRY(gemm(s, gd(El, 0, k.Da, 1, A, 0, (long long)k.d * k.Db, 1, s->X.p, 0, (long long)k.d * k.Db, 1,
                 k.Dp * k.wl, k.d * k.Db, k.Da, 1)));
  // the sparse G2 runs on the fp64 pipe; with the Ozaki contractions the dense
  // G2 (one batched GEMM with the MPO operand shared) is faster on the tensor cores
  if (sidx && sidx->p && s->oz_slices == 0) {
    const int R = k.d * k.wr;
    const int* rp = static_cast<const int*>(sidx->p);
    int e = zsparse_g2(launch_of(s->ctx), zp(s->X), static_cast<z64*>(T), rp, rp + R + 1,
                       static_cast<const z64*>(sval->p), R, k.wl * k.d, k.Db, k.Dp);
    if (e != TEVO_EUNSUPPORTED) return e;
  }
  // G2: T_p[(s v), b] = Wg[(s v), (w s')] X_p[(w s'), b]
  TRY(gemm(s, gd(Wg, 0, (long long)k.wl * k.d, 1, s->X.p, (long long)k.wl * k.d * k.Db, k.Db, 1, T,
                 (long long)k.d * k.wr * k.Db, k.Db, 1, k.d * k.wr, k.Db, k.wl * k.d, k.Dp)));
  return 0;
}

// G3: column-major B = T Er^T
int apply64(tevo_mps s, const StepDims& k, const z64* Er, z64* Bc) {
  const int M = k.Dp * k.d;
  return gemm(s, gd(s->T.p, 0, (long long)k.wr * k.Db, 1, Er, 0, 1, (long long)k.wr * k.Db, Bc, 0, 1, M, M,
                    k.Dq, k.wr * k.Db, 1));
}

// G3': Enew[q, (v b)] = sum conj(Q)[(p s), q] T[(p s), (v b)], Q column-major (ld = Dp d)
int env64(tevo_mps s, const StepDims& k, const z64* Qc, z64* Enew) {
  const int M = k.Dp * k.d;
  return gemm(s, gd(Qc, 0, M, 1, s->T.p, 0, (long long)k.wr * k.Db, 1, Enew, 0, (long long)k.wr * k.Db, 1,
                    k.Dq, k.wr * k.Db, M, 1, /*conjA=*/1));
}

// QR of the column-major Bq (m x n) and explicit Q written back into Bq
int qr_q(tevo_mps s, int m, int n, bool keep_r) {
  Launch L = launch_of(s->ctx);
  int* qf = static_cast<int*>(s->qrflags.p);
  int e = TEVO_EUNSUPPORTED;
  if (qf && s->coop_qr) {
    s->qr_epoch = s->qr_epoch == 0x3fffffff ? 1 : s->qr_epoch + 1;
    e = qr64_factor_coop(L, zp(s->Bq), m, n, zp(s->V), zp(s->tau), zp(s->beta), s->red.p, qf + 1, s->qr_epoch, qf);
  }
  if (e == TEVO_EUNSUPPORTED)
    e = qr64_factor(L, zp(s->Bq), m, n, zp(s->V), zp(s->tau), zp(s->beta), static_cast<double*>(s->red.p));
  TRY(e);
  if (keep_r) TRY(qr64_extract_r(L, zp(s->Bq), zp(s->beta), m, n, zp(s->Rm)));
  return qr64_form_q(L, zp(s->V), zp(s->tau), m, n, zp(s->Bq), 1, m, s->qrwy.p);
}

// store a column-major (Dl d) x Dr matrix as the site tensor [Dl][d][Dr]
int store_right(tevo_mps s, const z64* Bc, z64* site, int Dl, int d, int Dr) {
  const int m = Dl * d;
  return copy2d64(launch_of(s->ctx), Bc, 1, m, site, Dr, 1, m, Dr);
}

// store a column-major (Dr d) x Dl matrix (mirrored chain) as the site tensor [Dl][d][Dr]
int store_left(tevo_mps s, const z64* Bc, z64* site, int Dl, int d, int Dr) {
  const int m = Dr * d;
  Launch L = launch_of(s->ctx);
  TRY(copy2d64(L, Bc, 1, m, zp(s->Atmp), Dl, 1, m, Dl));  // -> [Dr][d][Dl]
  return mirror_site64(L, zp(s->Atmp), site, Dr, d, Dl);
}

int workspace(tevo_mps s, tevo_mpo W) {
  tevo_ctx c = s->ctx;
  const int L = s->L, d = s->d;
  int wmax = 1;
  for (int i = 0; i < L; ++i) wmax = std::max({wmax, W->wl[i], W->wr[i]});
  if (s->env.p && s->wmax >= wmax) return 0;
  ++g_persist_gen;
  s->wmax = wmax;
  s->env_off.assign(L + 1, 0);
  size_t off = 0;
  for (int b = 0; b <= L; ++b) {
    s->env_off[b] = off;
    int wb = (b == 0 || b == L) ? 1 : W->wr[b - 1];
    size_t bytes = sizeof(z64) * (size_t)s->dims[b] * wb * s->dims[b];
    off += (bytes + 255) / 256 * 256;
  }
  TRY(ensure(c, s->env, off));
  size_t xt = 0, bq = 0;
  for (int i = 0; i < L; ++i) {
    size_t a = (size_t)s->dims[i] * W->wl[i] * d * s->dims[i + 1];
    size_t b2 = (size_t)s->dims[i + 1] * W->wr[i] * d * s->dims[i];
    xt = std::max({xt, a, b2});
    bq = std::max(bq, (size_t)s->dims[i] * d * s->dims[i + 1]);
  }
  TRY(ensure(c, s->X, sizeof(z64) * xt));
  TRY(ensure(c, s->T, sizeof(z64) * xt));
  TRY(ensure(c, s->Bq, sizeof(z64) * bq));
  TRY(ensure(c, s->V, sizeof(z64) * bq));
  TRY(ensure(c, s->Atmp, sizeof(z64) * bq));
  TRY(ensure(c, s->tau, sizeof(z64) * (size_t)(s->D * d + 8)));
  TRY(ensure(c, s->beta, sizeof(z64) * (size_t)(s->D * d + 8)));
  TRY(ensure(c, s->Rm, sizeof(z64) * (size_t)s->D * s->D + 64));
  TRY(ensure(c, s->gemm_ws, (size_t)48 << 20));
  TRY(ensure(c, s->red, sizeof(double) * 4096));
  TRY(ensure(c, s->qrwy, qr64_wy_bytes(s->D * d)));
  if (!s->qrflags.p) {
    TRY(ensure(c, s->qrflags, sizeof(int) * ((size_t)s->D * d + 64)));
    TRYCUDA(cudaMemsetAsync(s->qrflags.p, 0, s->qrflags.bytes, c->stream));
    s->qr_epoch = 0;
  }
  return 0;
}

// LQ sweep from site L-1 down to 1 on the mirrored chain (Householder QR of
// the transposed site, R^T absorbed into the left neighbour)
int right_canonicalize(tevo_mps s, std::vector<Buf>& t) {
  Launch L = launch_of(s->ctx);
  const int d = s->d;
  for (int i = s->L - 1; i >= 1; --i) {
    const int Dl = s->dims[i], Dr = s->dims[i + 1];
    const int m = Dr * d, n = Dl;
    // mirrored site as a column-major m x n matrix: element ((r s), l) = A[l][s][r]
    TRY(mirror_site64(L, zp(t[i]), zp(s->Atmp), Dl, d, Dr));          // [Dr][d][Dl] = row-major m x n
    TRY(copy2d64(L, zp(s->Atmp), n, 1, zp(s->Bq), 1, m, m, n));       // -> column-major
    TRY(qr_q(s, m, n, true));
    TRY(store_left(s, zp(s->Bq), zp(t[i]), Dl, d, Dr));
    // left neighbour: A'[a][s][k] = sum_l A[a][s][l] R[k][l]
    const int Dll = s->dims[i - 1];
    TRY(gemm(s, gd(t[i - 1].p, 0, Dl, 1, s->Rm.p, 0, 1, n, s->Atmp.p, 0, n, 1, Dll * d, n, Dl, 1)));
    TRY(copy2d64(L, zp(s->Atmp), n, 1, zp(t[i - 1]), n, 1, Dll * d, n));
  }
  return 0;
}

StepDims right_dims(tevo_mps s, tevo_mpo W, int i) {
  return StepDims{s->dims[i], s->dims[i], W->wl[i], s->d, s->dims[i + 1], s->dims[i + 1], W->wr[i]};
}
StepDims left_dims(tevo_mps s, tevo_mpo W, int i) {
  return StepDims{s->dims[i + 1], s->dims[i + 1], W->wr[i], s->d, s->dims[i], s->dims[i], W->wl[i]};
}

// one fp64 sweep (rightward over 0..L-2, then leftward over L-1..1)
int sweep64(tevo_mps s, tevo_mpo W) {
  Launch L = launch_of(s->ctx);
  const int d = s->d;
  for (int i = 0; i + 1 < s->L; ++i) {
    StepDims k = right_dims(s, W, i);
    TRY(make_T64(s, k, env_slot(s, i), zp(s->A[i]), zp(W->Wr[i]), &W->Sr_idx[i], &W->Sr_val[i]));
    TRY(apply64(s, k, env_slot(s, i + 1), zp(s->Bq)));
    TRY(qr_q(s, k.Dp * d, k.Dq, false));
    TRY(store_right(s, zp(s->Bq), zp(s->Anew[i]), k.Dp, d, k.Dq));
    TRY(env64(s, k, zp(s->Bq), env_slot(s, i + 1)));
  }
  for (int i = s->L - 1; i >= 1; --i) {
    StepDims k = left_dims(s, W, i);
    TRY(mirror_site64(L, zp(s->A[i]), zp(s->Atmp), s->dims[i], d, s->dims[i + 1]));
    TRY(make_T64(s, k, env_slot(s, i + 1), zp(s->Atmp), zp(W->Wl[i]), &W->Sl_idx[i], &W->Sl_val[i]));
    TRY(apply64(s, k, env_slot(s, i), zp(s->Bq)));
    TRY(qr_q(s, k.Dp * d, k.Dq, false));
    TRY(store_left(s, zp(s->Bq), zp(s->Anew[i]), k.Dq, d, k.Dp));
    TRY(env64(s, k, zp(s->Bq), env_slot(s, i)));
  }
  return 0;
}

// ---------------------------------------------------------------------------
// two-site fit: the pair (i, i+1) in the rightward layout (rightward = true:
// site i keeps the leading left singular vectors of Theta) or the pair
// (i-1, i) on the mirrored chain (rightward = false: site i keeps them)
// ---------------------------------------------------------------------------
int two_site_workspace(tevo_mps s, tevo_mpo W) {
  tevo_ctx c = s->ctx;
  const int d = s->d;
  size_t xt = 0, md = 0;
  for (int i = 0; i < s->L; ++i) {
    xt = std::max({xt, (size_t)s->dims[i] * W->wl[i] * d * s->dims[i + 1],
                   (size_t)s->dims[i + 1] * W->wr[i] * d * s->dims[i]});
    md = std::max(md, (size_t)s->dims[i] * d);
  }
  md = std::max(md, (size_t)s->dims[s->L] * d);
  TRY(ensure(c, s->T2, sizeof(z64) * xt));
  TRY(ensure(c, s->Th, sizeof(z64) * md * (md + 1)));
  TRY(ensure(c, s->jac, jacobi_ws_bytes((int)md + 1)));
  return 0;
}

int two_site_update(tevo_mps s, tevo_mpo W, int i, bool rightward) {
  Launch L = launch_of(s->ctx);
  const int d = s->d;
  // kA: the site that keeps the singular vectors; kB: its partner (mirrored layout)
  StepDims kA, kB;
  const z64 *envA, *envB;
  if (rightward) {
    kA = right_dims(s, W, i);
    kB = left_dims(s, W, i + 1);
    TRY(make_T64(s, kA, env_slot(s, i), zp(s->A[i]), zp(W->Wr[i]), &W->Sr_idx[i], &W->Sr_val[i]));
    TRY(mirror_site64(L, zp(s->A[i + 1]), zp(s->Atmp), s->dims[i + 1], d, s->dims[i + 2]));
    TRY(make_T64(s, kB, env_slot(s, i + 2), zp(s->Atmp), zp(W->Wl[i + 1]), &W->Sl_idx[i + 1], &W->Sl_val[i + 1],
                 s->T2.p));
    envA = env_slot(s, i + 1);
    envB = nullptr;
  } else {
    kA = left_dims(s, W, i);
    kB = right_dims(s, W, i - 1);
    TRY(mirror_site64(L, zp(s->A[i]), zp(s->Atmp), s->dims[i], d, s->dims[i + 1]));
    TRY(make_T64(s, kA, env_slot(s, i + 1), zp(s->Atmp), zp(W->Wl[i]), &W->Sl_idx[i], &W->Sl_val[i]));
    TRY(make_T64(s, kB, env_slot(s, i - 1), zp(s->A[i - 1]), zp(W->Wr[i - 1]), &W->Sr_idx[i - 1],
                 &W->Sr_val[i - 1], s->T2.p));
    envA = env_slot(s, i);
    envB = nullptr;
  }
  (void)envB;
  // Theta[(p s), (q s')] = sum_(v b) T[(p s), (v b)] T2[(q s'), (v b)], column-major (ld = M)
  const int M = kA.Dp * d, N = kB.Dp * d, K = kA.wr * kA.Db;
  if (kB.wr * kB.Db != K) return TEVO_ESHAPE;
  const int Np = N + (N & 1);  // the Jacobi pairs columns: an odd count gets a zero column
  if (Np > N) TRY(fill64(L, zp(s->Th) + (size_t)N * M, (size_t)M, 0.0, 0.0));
  TRY(gemm(s, gd(s->T.p, 0, K, 1, s->T2.p, 0, 1, K, s->Th.p, 0, 1, M, M, N, K, 1)));
  const int k = kA.Dq;
  int* jerr = reinterpret_cast<int*>(scal(s, 6));
  TRY(jacobi_top_columns(L, zp(s->Th), M, Np, k, zp(s->Bq), s->jac.p, jerr));
  TRY(qr_q(s, M, k, false));
  if (rightward) {
    TRY(store_right(s, zp(s->Bq), zp(s->Anew[i]), kA.Dp, d, k));
  } else {
    TRY(store_left(s, zp(s->Bq), zp(s->Anew[i]), k, d, kA.Dp));
  }
  return env64(s, kA, zp(s->Bq), const_cast<z64*>(envA));
}

int sweep_two_site(tevo_mps s, tevo_mpo W) {
  for (int i = 0; i + 1 < s->L; ++i) TRY(two_site_update(s, W, i, true));
  for (int i = s->L - 1; i >= 1; --i) TRY(two_site_update(s, W, i, false));
  return 0;
}

// right environments of <bra|W|ket> for bonds L-1..1 (slot L holds 1)
int build_right_envs64(tevo_mps s, tevo_mpo W, std::vector<Buf>& bra, std::vector<Buf>& ket) {
  Launch L = launch_of(s->ctx);
  const int d = s->d;
  for (int i = s->L - 1; i >= 1; --i) {
    StepDims k = left_dims(s, W, i);
    TRY(mirror_site64(L, zp(ket[i]), zp(s->Atmp), s->dims[i], d, s->dims[i + 1]));
    TRY(make_T64(s, k, env_slot(s, i + 1), zp(s->Atmp), zp(W->Wl[i]), &W->Sl_idx[i], &W->Sl_val[i]));
    // bra^T as a column-major (Dr d) x Dl matrix
    TRY(mirror_site64(L, zp(bra[i]), zp(s->Atmp), s->dims[i], d, s->dims[i + 1]));
    TRY(copy2d64(L, zp(s->Atmp), k.Dq, 1, zp(s->Bq), 1, k.Dp * d, k.Dp * d, k.Dq));
    TRY(env64(s, k, zp(s->Bq), env_slot(s, i)));
  }
  return 0;
}

int centre64(tevo_mps s, tevo_mpo W) {
  Launch L = launch_of(s->ctx);
  const int d = s->d;
  StepDims k = left_dims(s, W, 0);
  TRY(mirror_site64(L, zp(s->A[0]), zp(s->Atmp), s->dims[0], d, s->dims[1]));
  TRY(make_T64(s, k, env_slot(s, 1), zp(s->Atmp), zp(W->Wl[0]), &W->Sl_idx[0], &W->Sl_val[0]));
  TRY(apply64(s, k, env_slot(s, 0), zp(s->Bq)));
  TRY(store_left(s, zp(s->Bq), zp(s->Anew[0]), k.Dq, d, k.Dp));
  return 0;
}

int finish_step(tevo_mps s) {
  Launch L = launch_of(s->ctx);
  const size_t n0 = (size_t)s->dims[0] * s->d * s->dims[1];
  TRY(norm2_64(L, zp(s->Anew[0]), n0, scal(s, 1), static_cast<double*>(s->red.p)));
  TRY(normalize64(L, zp(s->Anew[0]), n0, scal(s, 1), scal(s, 0), reinterpret_cast<int*>(scal(s, 4))));
  std::swap(s->A, s->Anew);
  s->parity ^= 1;
  s->canonical = true;
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int tevo_ctx_create(void* stream, tevo_ctx* out) {
  if (!out) return TEVO_EINVAL;
  tevo_ctx c = new (std::nothrow) tevo_ctx_s;
  if (!c) return TEVO_ENOMEM;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return TEVO_ECUDA;
  }
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return TEVO_ECUDA;
  }
  *out = c;
  return 0;
}

extern "C" int tevo_ctx_destroy(tevo_ctx c) {
  if (!c) return TEVO_EINVAL;
  for (auto& r : c->prof.recs) {
    cudaEventDestroy(reinterpret_cast<cudaEvent_t>(r.e0));
    cudaEventDestroy(reinterpret_cast<cudaEvent_t>(r.e1));
  }
  for (void* e : c->prof.pool) cudaEventDestroy(reinterpret_cast<cudaEvent_t>(e));
  delete c;
  return 0;
}

extern "C" int tevo_ctx_set_allocator(tevo_ctx c, tevo_alloc_fn a, tevo_free_fn f, void* user) {
  if (!c || (a == nullptr) != (f == nullptr)) return TEVO_EINVAL;
  c->alloc = a;
  c->free_fn = f;
  c->user = user;
  return 0;
}

extern "C" int tevo_ctx_set_stream(tevo_ctx c, void* stream) {
  if (!c) return TEVO_EINVAL;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return 0;
}

extern "C" int tevo_launch_count(tevo_ctx c, long long* count, int reset) {
  if (!c || !count) return TEVO_EINVAL;
  *count = c->launches;
  if (reset) c->launches = 0;
  return 0;
}

namespace tevo {
int Prof::begin(cudaStream_t s, int cls, double flops, double bytes) {
  if (!on) return -1;
  auto get = [&]() -> void* {
    if (!pool.empty()) {
      void* e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  };
  void* e0 = get();
  void* e1 = get();
  if (!e0 || !e1) return -1;
  cudaEventRecord(reinterpret_cast<cudaEvent_t>(e0), s);
  recs.push_back(Rec{cls, e0, e1, flops, bytes});
  return int(recs.size()) - 1;
}
void Prof::end(cudaStream_t s, int idx) {
  if (idx < 0) return;
  cudaEventRecord(reinterpret_cast<cudaEvent_t>(recs[idx].e1), s);
}
}  // namespace tevo

extern "C" int tevo_prof_enable(tevo_ctx c, int enable) {
  if (!c) return TEVO_EINVAL;
  c->prof.on = enable != 0;
  return 0;
}

extern "C" int tevo_prof_read(tevo_ctx c, int cls, double* ms, long long* n, double* flops, double* bytes) {
  if (!c || !ms || !n || !flops || !bytes || cls < 0 || cls >= TEVO_PROF_CLASSES) return TEVO_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TEVO_ECUDA;
  *ms = 0;
  *n = 0;
  *flops = 0;
  *bytes = 0;
  std::vector<Prof::Rec> keep;
  for (auto& r : c->prof.recs) {
    if (r.cls != cls) {
      keep.push_back(r);
      continue;
    }
    float t = 0;
    if (cudaEventElapsedTime(&t, reinterpret_cast<cudaEvent_t>(r.e0), reinterpret_cast<cudaEvent_t>(r.e1)) !=
        cudaSuccess)
      return TEVO_ECUDA;
    *ms += t;
    *n += 1;
    *flops += r.flops;
    *bytes += r.bytes;
    c->prof.pool.push_back(r.e0);
    c->prof.pool.push_back(r.e1);
  }
  c->prof.recs.swap(keep);
  return 0;
}

extern "C" const char* tevo_strerror(int code) {
  switch (code) {
    case TEVO_OK: return "ok";
    case TEVO_EINVAL: return "invalid argument";
    case TEVO_ESHAPE: return "shape mismatch";
    case TEVO_ETAU: return "tau differs from the MPO's tau";
    case TEVO_ENOMEM: return "out of memory";
    case TEVO_ECUDA: return "CUDA error";
    case TEVO_ENONFINITE: return "non-finite norm";
    case TEVO_ETIMEOUT: return "device wait timed out";
    case TEVO_EUNSUPPORTED: return "unsupported";
    default: return "unknown error";
  }
}

// ---------------------------------------------------------------------------
// MPO
// ---------------------------------------------------------------------------
extern "C" int mpo_build(tevo_ctx c, int L, int d, int chi, const double* A, const double* B, const double* C,
                         const double* Dh, int N, double tau_re, double tau_im, int variant, tevo_mpo* out) {
  if (!c || !A || !B || !C || !Dh || !out) return TEVO_EINVAL;
  if (L < 2 || d < 1 || chi < 1 || N < 1 || N > 6 || variant < 0 || variant > 3) return TEVO_EINVAL;
  if (!std::isfinite(tau_re) || !std::isfinite(tau_im)) return TEVO_EINVAL;
  tevo_mpo W = new (std::nothrow) tevo_mpo_s;
  if (!W) return TEVO_ENOMEM;
  W->ctx = c;
  W->L = L;
  W->d = d;
  W->chi = chi;
  W->N = N;
  W->variant = variant;
  W->tau_re = tau_re;
  W->tau_im = tau_im;
  try {
    build_mpo_host(L, d, chi, A, B, C, Dh, N, tau_re, tau_im, variant, W->host, W->wl, W->wr);
  } catch (...) {
    delete W;
    return TEVO_ENOMEM;
  }
  W->W.resize(L);
  W->Wr.resize(L);
  W->Wl.resize(L);
  W->Sr_idx.resize(L);
  W->Sr_val.resize(L);
  W->Sl_idx.resize(L);
  W->Sl_val.resize(L);
  for (int i = 0; i < L; ++i) {
    const int wl = W->wl[i], wr = W->wr[i];
    const auto& S = W->host[i];
    std::vector<std::complex<double>> gr((size_t)d * wr * wl * d), gl((size_t)d * wl * wr * d);
    for (int a = 0; a < wl; ++a)
      for (int s = 0; s < d; ++s)
        for (int t = 0; t < d; ++t)
          for (int b = 0; b < wr; ++b) {
            auto v = S[((size_t(a) * d + s) * d + t) * wr + b];
            gr[((size_t)s * wr + b) * (wl * d) + (size_t)a * d + t] = v;  // [(s wr)][(wl s')]
            gl[((size_t)s * wl + a) * (wr * d) + (size_t)b * d + t] = v;  // [(s wl)][(wr s')]
          }
    const size_t bytes = sizeof(z64) * S.size();
    // CSR of the two G2 operands: rows d*wr (d*wl), columns wl*d (wr*d)
    auto csr = [&](const std::vector<std::complex<double>>& g, int rows, int cols, Buf& bidx, Buf& bval) -> int {
      std::vector<int> idx(1, 0);
      std::vector<std::complex<double>> val;
      std::vector<int> cidx;
      for (int r = 0; r < rows; ++r) {
        for (int q = 0; q < cols; ++q) {
          auto v = g[(size_t)r * cols + q];
          if (v != std::complex<double>(0.0, 0.0)) {
            cidx.push_back(q);
            val.push_back(v);
          }
        }
        idx.push_back((int)cidx.size());
      }
      idx.insert(idx.end(), cidx.begin(), cidx.end());
      if (val.empty()) val.push_back(0.0);
      int e = dalloc(c, bidx, sizeof(int) * idx.size());
      if (!e) e = dalloc(c, bval, sizeof(z64) * val.size());
      if (e) return e;
      if (cudaMemcpyAsync(bidx.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, c->stream) !=
              cudaSuccess ||
          cudaMemcpyAsync(bval.p, val.data(), sizeof(z64) * val.size(), cudaMemcpyHostToDevice, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return TEVO_ECUDA;
      return 0;
    };
    int e = csr(gr, d * wr, wl * d, W->Sr_idx[i], W->Sr_val[i]);
    if (!e) e = csr(gl, d * wl, wr * d, W->Sl_idx[i], W->Sl_val[i]);
    if (e) {
      mpo_destroy(W);
      return e;
    }
    e = dalloc(c, W->W[i], bytes);
    if (!e) e = dalloc(c, W->Wr[i], bytes);
    if (!e) e = dalloc(c, W->Wl[i], bytes);
    if (e) {
      mpo_destroy(W);
      return e;
    }
    if (cudaMemcpyAsync(W->W[i].p, S.data(), bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(W->Wr[i].p, gr.data(), bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(W->Wl[i].p, gl.data(), bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      mpo_destroy(W);
      return TEVO_ECUDA;
    }
  }
  *out = W;
  return 0;
}

extern "C" int mpo_build_host(int L, int d, int chi, const double* A, const double* B, const double* C,
                              const double* Dh, int N, double tau_re, double tau_im, int variant, int* w_out,
                              double* W_out, size_t* count) {
  if (!A || !B || !C || !Dh || !w_out || !count) return TEVO_EINVAL;
  if (L < 2 || d < 1 || chi < 1 || N < 1 || N > 6 || variant < 0 || variant > 3) return TEVO_EINVAL;
  std::vector<std::vector<std::complex<double>>> sites;
  std::vector<int> wl, wr;
  try {
    build_mpo_host(L, d, chi, A, B, C, Dh, N, tau_re, tau_im, variant, sites, wl, wr);
  } catch (...) {
    return TEVO_ENOMEM;
  }
  size_t total = 0;
  for (auto& v : sites) total += v.size();
  w_out[0] = wl[0];
  for (int i = 0; i < L; ++i) w_out[i + 1] = wr[i];
  if (W_out) {
    if (*count < total) return TEVO_EINVAL;
    size_t off = 0;
    for (auto& v : sites) {
      std::memcpy(W_out + 2 * off, v.data(), sizeof(z64) * v.size());
      off += v.size();
    }
  }
  *count = total;
  return 0;
}

extern "C" int mpo_bond_dims(tevo_mpo W, int* w) {
  if (!W || !w) return TEVO_EINVAL;
  w[0] = W->wl[0];
  for (int i = 0; i < W->L; ++i) w[i + 1] = W->wr[i];
  return 0;
}

extern "C" int mpo_get_site(tevo_mpo W, int i, double* out) {
  if (!W || !out || i < 0 || i >= W->L) return TEVO_EINVAL;
  std::memcpy(out, W->host[i].data(), sizeof(z64) * W->host[i].size());
  return 0;
}

extern "C" int mpo_destroy(tevo_mpo W) {
  if (!W) return TEVO_EINVAL;
  for (auto& b : W->W) dfree(W->ctx, b);
  for (auto& b : W->Wr) dfree(W->ctx, b);
  for (auto& b : W->Wl) dfree(W->ctx, b);
  for (auto* v : {&W->Sr_idx, &W->Sr_val, &W->Sl_idx, &W->Sl_val})
    for (auto& b : *v) dfree(W->ctx, b);
  mixed_mpo_destroy(W->ctx, W->mixed);
  delete W;
  return 0;
}

// ---------------------------------------------------------------------------
// MPS
// ---------------------------------------------------------------------------
extern "C" int mps_init(tevo_ctx c, int L, int d, int D, const double* v, tevo_mps* out) {
  if (!c || !v || !out || L < 2 || d < 1 || D < 1) return TEVO_EINVAL;
  tevo_mps s = new (std::nothrow) tevo_mps_s;
  if (!s) return TEVO_ENOMEM;
  s->ctx = c;
  s->L = L;
  s->d = d;
  s->D = D;
  s->dims.resize(L + 1);
  for (int i = 0; i <= L; ++i) {
    long long p = 1;
    for (int k = 0; k < std::min(i, L - i) && p < D; ++k) p = std::min<long long>(p * d, D);
    s->dims[i] = int(p);
  }
  s->A.resize(L);
  s->Anew.resize(L);
  int e = dalloc(c, s->scalars, sizeof(double) * 16);
  for (int i = 0; i < L && !e; ++i) {
    const size_t n = (size_t)s->dims[i] * d * s->dims[i + 1];
    e = dalloc(c, s->A[i], sizeof(z64) * n);
    if (!e) e = dalloc(c, s->Anew[i], sizeof(z64) * n);
    if (!e) {
      std::vector<z64> h(n, z64{0, 0});
      for (int t = 0; t < d; ++t) h[(size_t)t * s->dims[i + 1]] = z64{v[2 * ((size_t)i * d + t)], v[2 * ((size_t)i * d + t) + 1]};
      if (cudaMemcpyAsync(s->A[i].p, h.data(), sizeof(z64) * n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        e = TEVO_ECUDA;
    }
  }
  if (!e) {
    double z[16] = {0};
    if (cudaMemcpyAsync(s->scalars.p, z, sizeof(z), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      e = TEVO_ECUDA;
  }
  if (e) {
    mps_destroy(s);
    return e;
  }
  *out = s;
  return 0;
}

extern "C" int mps_bond_dims(tevo_mps s, int* out) {
  if (!s || !out) return TEVO_EINVAL;
  for (int i = 0; i <= s->L; ++i) out[i] = s->dims[i];
  return 0;
}

extern "C" int mps_get_site(tevo_mps s, int i, double* out) {
  if (!s || !out || i < 0 || i >= s->L) return TEVO_EINVAL;
  const size_t n = (size_t)s->dims[i] * s->d * s->dims[i + 1];
  if (cudaMemcpyAsync(out, s->A[i].p, sizeof(z64) * n, cudaMemcpyDeviceToHost, s->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->ctx->stream) != cudaSuccess)
    return TEVO_ECUDA;
  return 0;
}

extern "C" int mps_set_site(tevo_mps s, int i, const double* in) {
  if (!s || !in || i < 0 || i >= s->L) return TEVO_EINVAL;
  const size_t n = (size_t)s->dims[i] * s->d * s->dims[i + 1];
  if (cudaMemcpyAsync(s->A[i].p, in, sizeof(z64) * n, cudaMemcpyHostToDevice, s->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->ctx->stream) != cudaSuccess)
    return TEVO_ECUDA;
  s->canonical = false;
  return 0;
}

extern "C" int mps_log_norm(tevo_mps s, double* out) {
  if (!s || !out) return TEVO_EINVAL;
  if (cudaMemcpyAsync(out, scal(s, 0), sizeof(double), cudaMemcpyDeviceToHost, s->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->ctx->stream) != cudaSuccess)
    return TEVO_ECUDA;
  return 0;
}

extern "C" int mps_destroy(tevo_mps s) {
  if (!s) return TEVO_EINVAL;
  tevo_ctx c = s->ctx;
  for (auto& b : s->A) dfree(c, b);
  for (auto& b : s->Anew) dfree(c, b);
  for (Buf* b : {&s->scalars, &s->env, &s->X, &s->T, &s->Bq, &s->V, &s->tau, &s->beta, &s->Atmp, &s->Rm,
                 &s->gemm_ws, &s->red, &s->qrflags, &s->qrwy, &s->T2, &s->Th, &s->jac, &s->oz_ws})
    dfree(c, *b);
  mixed_state_destroy(c, s->mixed);
  delete s;
  return 0;
}

// ---------------------------------------------------------------------------
// evolve_step
// ---------------------------------------------------------------------------
namespace {

// slice count of an Ozaki precision flag (0 when the flag is absent, -1 when invalid)
int oz_slices_of(int precision) {
  if (!(precision & TEVO_OZAKI)) return (precision >> 12) ? -1 : 0;
  const int g = (precision >> 12) & 0xF;
  if (precision >> 16) return -1;
  if (g == 0) return 8;
  return g <= oz_max_slices() ? g : -1;
}

int strip_oz(int precision) { return precision & ~(TEVO_OZAKI | (0xF << 12)); }

int check_step_args(tevo_mps s, tevo_mpo W, int sweeps, int precision) {
  if (!s || !W || sweeps < 1) return TEVO_EINVAL;
  // the two-site fit: the fp64 form only (its contractions may be Ozaki GEMMs)
  if (precision & TEVO_TWO_SITE) {
    if ((strip_oz(precision) & ~TEVO_TWO_SITE) != TEVO_FP64) return TEVO_EINVAL;
    precision &= ~TEVO_TWO_SITE;
  }
  const int oz = oz_slices_of(precision);
  if (oz < 0) return TEVO_EINVAL;
  precision = strip_oz(precision);
  const bool tc_only = (precision & TEVO_TC_ONLY) != 0;
  if (tc_only && oz) return TEVO_EINVAL;
  precision &= ~TEVO_TC_ONLY;
  if (precision < TEVO_FP64 || precision > TEVO_BF16X3) return TEVO_EINVAL;
  if (tc_only && precision == TEVO_FP64) return TEVO_EINVAL;
  if (W->L != s->L || W->d != s->d) return TEVO_ESHAPE;
  return 0;
}

// issue one time step on the context stream; no host synchronisation (so it can
// be captured in a CUDA graph once the workspaces exist)
int evolve_issue_body(tevo_mps s, tevo_mpo W, int sweeps, int precision, bool* mixed_out);

int evolve_issue(tevo_mps s, tevo_mpo W, int sweeps, int precision, bool* mixed_out) {
  s->two_site = (precision & TEVO_TWO_SITE) != 0;
  precision &= ~TEVO_TWO_SITE;
  const int oz = oz_slices_of(precision);
  if (oz < 0) return TEVO_EINVAL;
  if (oz && cudaMemsetAsync(scal(s, OZ_FLAG_SLOT), 0, sizeof(double), s->ctx->stream) != cudaSuccess)
    return TEVO_ECUDA;
  // the fp64 contractions of this step only (measure_local / mps_overlap stay native)
  s->oz_slices = oz;
  const int e = evolve_issue_body(s, W, sweeps, strip_oz(precision), mixed_out);
  s->oz_slices = 0;
  return e;
}

int evolve_issue_body(tevo_mps s, tevo_mpo W, int sweeps, int precision, bool* mixed_out) {
  const bool tc_only = (precision & TEVO_TC_ONLY) != 0;
  precision &= ~TEVO_TC_ONLY;
  tevo_ctx c = s->ctx;
  TRY(workspace(s, W));
  Launch L = launch_of(c);
  const int d = s->d;
  TRY(fill64(L, env_slot(s, 0), 1, 1.0, 0.0));
  TRY(fill64(L, env_slot(s, s->L), 1, 1.0, 0.0));
  // bra of the first environments: phi0 = psi, made right-canonical when psi is not
  std::vector<Buf>* bra = &s->A;
  if (!s->canonical) {
    for (int i = 0; i < s->L; ++i) {
      const size_t n = (size_t)s->dims[i] * d * s->dims[i + 1];
      TRYCUDA(cudaMemcpyAsync(s->Anew[i].p, s->A[i].p, sizeof(z64) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    TRY(right_canonicalize(s, s->Anew));
    bra = &s->Anew;
  }
  const bool mixed = precision != TEVO_FP64 && (sweeps > 1 || tc_only);
  if (mixed) {
    TRY(mixed_prepare(c, W, s, precision));
    TRY(mixed_build_right_envs(c, W, s, bra == &s->Anew, precision));
    const int nlp = tc_only ? sweeps : sweeps - 1;
    for (int k = 0; k < nlp; ++k) TRY(mixed_sweep(c, W, s, precision));
    if (!tc_only) {
      // fp64 rebuild of the right environments from the fitted phi, then one fp64 sweep
      TRY(build_right_envs64(s, W, s->Anew, s->A));
    }
  } else {
    TRY(build_right_envs64(s, W, *bra, s->A));
  }
  if (tc_only) {
    TRY(mixed_centre(c, W, s, precision));
  } else {
    const int n64 = mixed ? 1 : sweeps;
    if (s->two_site) {
      TRY(two_site_workspace(s, W));
      TRYCUDA(cudaMemsetAsync(scal(s, 6), 0, sizeof(double), c->stream));
      for (int k = 0; k < n64; ++k) TRY(sweep_two_site(s, W));
    } else {
      for (int k = 0; k < n64; ++k) TRY(sweep64(s, W));
    }
    TRY(centre64(s, W));
  }
  TRY(finish_step(s));
  *mixed_out = mixed;
  return cudaGetLastError() == cudaSuccess ? 0 : TEVO_ECUDA;
}

// device flags of the step just issued (synchronises the context stream)
int evolve_check(tevo_mps s, bool mixed) {
  tevo_ctx c = s->ctx;
  int flag = 0, tflag = 0, qflag = 0, oflag = 0, jflag = 0;
  TRYCUDA(cudaMemcpyAsync(&flag, scal(s, 4), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (s->two_site) TRYCUDA(cudaMemcpyAsync(&jflag, scal(s, 6), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TRYCUDA(cudaMemcpyAsync(&oflag, scal(s, OZ_FLAG_SLOT), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (s->qrflags.p)
    TRYCUDA(cudaMemcpyAsync(&qflag, s->qrflags.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (mixed) TRY(mixed_error_flag(c, s, &tflag));
  TRYCUDA(cudaStreamSynchronize(c->stream));
  if (tflag || qflag || oflag || jflag) return TEVO_ETIMEOUT;
  if (flag) return TEVO_ENONFINITE;
  return 0;
}

}  // namespace

extern "C" int evolve_step(tevo_mps s, tevo_mpo W, double tau_re, double tau_im, int D, int sweeps, int precision) {
  TRY(check_step_args(s, W, sweeps, precision));
  if (D != s->D) return TEVO_ESHAPE;
  if (tau_re != W->tau_re || tau_im != W->tau_im) return TEVO_ETAU;
  bool mixed = false;
  TRY(evolve_issue(s, W, sweeps, precision, &mixed));
  return evolve_check(s, mixed);
}

// ---------------------------------------------------------------------------
// batched form: independent chains stepped together
// ---------------------------------------------------------------------------
namespace {

struct BatchPlan {
  std::vector<tevo_mps> psis;
  std::vector<tevo_mpo> Ws;
  int sweeps = 0, precision = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;  // stream the graph is captured on and launched from
  std::vector<int> order;         // issue order of the chains
  int nstreams = 0;
  int tune_next = 0;              // index into the candidate list while tuning
  std::vector<std::pair<int, float>> tuned;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  long long graph_launches[2] = {0, 0};
  long long gen[2] = {-1, -1};  // g_persist_gen at capture
  bool mixed = false;
};

BatchPlan* g_plan_cache = nullptr;  // one plan per process (the last batch used)

void plan_free(BatchPlan* p) {
  if (!p) return;
  for (auto& e : p->exec)
    if (e) cudaGraphExecDestroy(e);
  for (auto& st : p->streams) cudaStreamDestroy(st);
  for (auto& ev : p->done) cudaEventDestroy(ev);
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->origin) cudaStreamDestroy(p->origin);
  delete p;
}

// work of one chain step (useful MACs), for the largest-first issue order
double chain_work(tevo_mps s, tevo_mpo W) {
  double w = 0;
  for (int i = 0; i < s->L; ++i)
    w += (double)s->dims[i] * s->dims[i + 1] * (s->dims[i] + s->dims[i + 1]) * W->wr[i];
  return w;
}

int plan_streams(BatchPlan* p, int nstreams) {
  while ((int)p->streams.size() < nstreams) {
    cudaStream_t st;
    cudaEvent_t ev;
    TRYCUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    TRYCUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    p->streams.push_back(st);
    p->done.push_back(ev);
  }
  p->nstreams = nstreams;
  return 0;
}

// issue every chain's step on the worker streams, forked from and joined into origin
int batch_issue(BatchPlan* p, cudaStream_t origin) {
  TRYCUDA(cudaEventRecord(p->fork, origin));
  for (int k = 0; k < p->nstreams; ++k) TRYCUDA(cudaStreamWaitEvent(p->streams[k], p->fork, 0));
  for (size_t j = 0; j < p->order.size(); ++j) {
    const int c = p->order[j];
    tevo_mps s = p->psis[c];
    cudaStream_t saved = s->ctx->stream;
    s->ctx->stream = p->streams[j % p->nstreams];
    s->coop_qr = false;
    bool mixed = false;
    int e = evolve_issue(s, p->Ws[c], p->sweeps, p->precision, &mixed);
    s->coop_qr = true;
    s->ctx->stream = saved;
    if (e) return e;
    p->mixed = mixed;
  }
  for (int k = 0; k < p->nstreams; ++k) {
    TRYCUDA(cudaEventRecord(p->done[k], p->streams[k]));
    TRYCUDA(cudaStreamWaitEvent(origin, p->done[k], 0));
  }
  return 0;
}

int batch_check(BatchPlan* p) {
  for (size_t c = 0; c < p->psis.size(); ++c) {
    tevo_mps s = p->psis[c];
    int flag = 0, tflag = 0;
    TRYCUDA(cudaMemcpy(&flag, scal(s, 4), sizeof(int), cudaMemcpyDeviceToHost));
    if (p->mixed) {
      TRY(mixed_error_flag(s->ctx, s, &tflag));
      TRYCUDA(cudaStreamSynchronize(s->ctx->stream));
    }
    if (tflag) return TEVO_ETIMEOUT;
    if (flag) return TEVO_ENONFINITE;
  }
  return 0;
}

}  // namespace

extern "C" int evolve_step_batched(tevo_mps* psis, const tevo_mpo* Ws, int n, int sweeps, int precision) {
  if (!psis || !Ws || n < 1) return TEVO_EINVAL;
  for (int c = 0; c < n; ++c) TRY(check_step_args(psis[c], Ws[c], sweeps, precision));
  if (oz_slices_of(precision) != 0) return TEVO_EUNSUPPORTED;  // the Ozaki form is single-chain only
  if (precision & TEVO_TWO_SITE) return TEVO_EUNSUPPORTED;     // so is the two-site fit
  for (int c = 0; c < n; ++c)
    for (int k = c + 1; k < n; ++k)
      if (psis[c] == psis[k]) return TEVO_EINVAL;
  tevo_ctx c0 = psis[0]->ctx;
  // reuse the cached plan when the batch is the same
  BatchPlan* p = g_plan_cache;
  bool same = p && p->sweeps == sweeps && p->precision == precision && (int)p->psis.size() == n;
  for (int c = 0; same && c < n; ++c) same = p->psis[c] == psis[c] && p->Ws[c] == Ws[c];
  if (!same) {
    plan_free(g_plan_cache);
    g_plan_cache = p = new BatchPlan;
    p->psis.assign(psis, psis + n);
    p->Ws.assign(Ws, Ws + n);
    p->sweeps = sweeps;
    p->precision = precision;
    TRYCUDA(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    TRYCUDA(cudaStreamCreateWithFlags(&p->origin, cudaStreamNonBlocking));
    p->order.resize(n);
    std::vector<double> work(n);
    for (int c = 0; c < n; ++c) {
      p->order[c] = c;
      work[c] = chain_work(psis[c], Ws[c]);
    }
    // largest chains first, so the longest dependency chains start earliest
    std::stable_sort(p->order.begin(), p->order.end(), [&](int a, int b) { return work[a] > work[b]; });
  }
  bool all_canonical = true;
  for (int c = 0; c < n; ++c) all_canonical = all_canonical && psis[c]->canonical;
  // the caller's stream orders the batch against its other work
  cudaStream_t caller = c0->stream;
  TRYCUDA(cudaEventRecord(p->fork, caller));
  TRYCUDA(cudaStreamWaitEvent(p->origin, p->fork, 0));
  // candidate schedules: worker-stream counts, tried once each (uncaptured, timed)
  const int cands[3] = {std::min(n, 64), std::min(n, 16), std::min(n, 4)};
  if (!all_canonical || p->tune_next < 3) {
    const int k = all_canonical ? p->tune_next : 0;
    TRY(plan_streams(p, cands[k]));
    cudaEvent_t t0, t1;
    TRYCUDA(cudaEventCreate(&t0));
    TRYCUDA(cudaEventCreate(&t1));
    TRYCUDA(cudaEventRecord(t0, p->origin));
    TRY(batch_issue(p, p->origin));
    TRYCUDA(cudaEventRecord(t1, p->origin));
    TRYCUDA(cudaEventSynchronize(t1));
    float ms = 0;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (all_canonical) {
      p->tuned.push_back({cands[k], ms});
      ++p->tune_next;
      if (p->tune_next == 3) {
        int best = p->tuned[0].first;
        float bms = p->tuned[0].second;
        for (auto& t : p->tuned)
          if (t.second < bms) {
            best = t.first;
            bms = t.second;
          }
        TRY(plan_streams(p, best));
      }
    }
  } else {
    // a captured step reads and writes the buffers of the parity it was captured at
    int par = psis[0]->parity;
    bool common = true;
    for (int c = 1; c < n; ++c) common = common && psis[c]->parity == par;
    for (int q = 0; q < 2; ++q)
      if (p->exec[q] && p->gen[q] != g_persist_gen) {
        cudaGraphExecDestroy(p->exec[q]);
        p->exec[q] = nullptr;
      }
    if (!common || c0->prof.on) {
      TRY(batch_issue(p, p->origin));
    } else if (!p->exec[par]) {
      cudaGraph_t g;
      const long long before = c0->launches;
      TRYCUDA(cudaStreamBeginCapture(p->origin, cudaStreamCaptureModeThreadLocal));
      int e = batch_issue(p, p->origin);  // swaps every chain's psi/phi (host side)
      cudaError_t ce = cudaStreamEndCapture(p->origin, &g);
      if (e) return e;
      if (ce != cudaSuccess) return TEVO_ECUDA;
      cudaError_t ie = cudaGraphInstantiate(&p->exec[par], g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        p->exec[par] = nullptr;
        return TEVO_ECUDA;
      }
      p->graph_launches[par] = c0->launches - before;
      p->gen[par] = g_persist_gen;
      TRYCUDA(cudaGraphLaunch(p->exec[par], p->origin));
    } else {
      // replay, repeating the host-side psi/phi swap of every chain
      for (int c = 0; c < n; ++c) {
        std::swap(psis[c]->A, psis[c]->Anew);
        psis[c]->parity ^= 1;
      }
      TRYCUDA(cudaGraphLaunch(p->exec[par], p->origin));
      c0->launches += p->graph_launches[par];
    }
  }
  TRYCUDA(cudaEventRecord(p->fork, p->origin));
  TRYCUDA(cudaStreamWaitEvent(caller, p->fork, 0));
  TRYCUDA(cudaStreamSynchronize(caller));
  return batch_check(p);
}

// accessors used by the mixed-precision translation unit
namespace tevo {
int mps_L(tevo_mps s) { return s->L; }
int mps_d(tevo_mps s) { return s->d; }
const std::vector<int>& mps_dims(tevo_mps s) { return s->dims; }
MixedState*& mps_mixed(tevo_mps s) { return s->mixed; }
MixedMPO*& mpo_mixed(tevo_mpo W) { return W->mixed; }
int mpo_wl(tevo_mpo W, int i) { return W->wl[i]; }
int mpo_wr(tevo_mpo W, int i) { return W->wr[i]; }
const void* mpo_dev_wr(tevo_mpo W, int i) { return W->Wr[i].p; }
const void* mpo_dev_wl(tevo_mpo W, int i) { return W->Wl[i].p; }
void* mps_site(tevo_mps s, int i, bool fresh) { return fresh ? s->Anew[i].p : s->A[i].p; }
void* mps_env_slot(tevo_mps s, int b) { return env_slot(s, b); }
void* mps_buf_T(tevo_mps s) { return s->T.p; }
void* mps_buf_X(tevo_mps s) { return s->X.p; }
void* mps_buf_Bq(tevo_mps s) { return s->Bq.p; }
void* mps_buf_Atmp(tevo_mps s) { return s->Atmp.p; }
int mps_qr_q(tevo_mps s, int m, int n) { return qr_q(s, m, n, false); }
int mps_store_right(tevo_mps s, int i) {
  return store_right(s, zp(s->Bq), zp(s->Anew[i]), s->dims[i], s->d, s->dims[i + 1]);
}
int mps_store_left(tevo_mps s, int i) {
  return store_left(s, zp(s->Bq), zp(s->Anew[i]), s->dims[i], s->d, s->dims[i + 1]);
}
int ctx_alloc(tevo_ctx c, void** p, size_t bytes) {
  Buf b;
  int e = dalloc(c, b, bytes);
  *p = b.p;
  return e;
}
void ctx_free(tevo_ctx c, void* p) {
  Buf b;
  b.p = p;
  b.bytes = 1;
  dfree(c, b);
}
Launch ctx_launch(tevo_ctx c) { return launch_of(c); }
}  // namespace tevo

// ---------------------------------------------------------------------------
// observables
// ---------------------------------------------------------------------------
extern "C" int measure_local(tevo_mps s, int nops, const double* ops, double* out) {
  if (!s || !ops || !out || nops < 1) return TEVO_EINVAL;
  tevo_ctx c = s->ctx;
  Launch Lc = launch_of(c);
  const int L = s->L, d = s->d;
  // transfer matrices: El[i] (bond i) from the left, Er[i] from the right, each [D_i][D_i]
  std::vector<size_t> off(L + 1);
  size_t tot = 0;
  for (int b = 0; b <= L; ++b) {
    off[b] = tot;
    tot += (size_t)s->dims[b] * s->dims[b];
  }
  size_t bq = 0;
  for (int i = 0; i < L; ++i) bq = std::max(bq, (size_t)s->dims[i] * d * s->dims[i + 1]);
  // a state left by evolve_step is right-canonical from site 1 on (its sites
  // are the isometries of the last leftward sweep): its right transfer
  // matrices are identities, and <O_i> needs only the site's density
  // rho_i[s][t] = sum conj(A_i[a0][s][a]) (El_i A_i)[a0][t][a] from the left
  // sweep (no per-operator contractions)
  const bool dens = s->canonical && d <= 4;
  Buf El, Er, Y, Z, Wm, OA, opsd, vals, part;
  int e = dalloc(c, El, sizeof(z64) * tot);
  if (!e && dens) e = dalloc(c, part, sizeof(z64) * rho_part_count(L, d));
  if (!e) e = dalloc(c, Er, sizeof(z64) * tot);
  if (!e) e = dalloc(c, Y, sizeof(z64) * bq);
  if (!e) e = dalloc(c, Z, sizeof(z64) * bq);
  if (!e) e = dalloc(c, OA, sizeof(z64) * bq);
  if (!e) e = dalloc(c, Wm, sizeof(z64) * (size_t)s->D * s->D + 16);
  if (!e) e = dalloc(c, opsd, sizeof(z64) * (size_t)nops * d * d);
  if (!e) e = dalloc(c, vals, sizeof(z64) * ((size_t)nops * L + 1));
  if (!e) e = ensure(c, s->gemm_ws, (size_t)48 << 20);
  if (!e) e = ensure(c, s->red, sizeof(double) * 4096);
  if (!e) e = ensure(c, s->Atmp, sizeof(z64) * bq);
  auto cleanup = [&]() {
    for (Buf* b : {&El, &Er, &Y, &Z, &Wm, &OA, &opsd, &vals, &part}) dfree(c, *b);
  };
  auto run = [&]() -> int {
    TRYCUDA(cudaMemcpyAsync(opsd.p, ops, sizeof(z64) * (size_t)nops * d * d, cudaMemcpyHostToDevice, c->stream));
    z64* el = zp(El);
    z64* er = zp(Er);
    TRY(fill64(Lc, el + off[0], 1, 1.0, 0.0));
    TRY(fill64(Lc, er + off[L], 1, 1.0, 0.0));
    // El[i+1][a][b] = sum conj(A[a0][s][a]) El[i][a0][b0] A[b0][s][b]
    for (int i = 0; i < L; ++i) {
      const int Dl = s->dims[i], Dr = s->dims[i + 1];
      TRY(gemm(s, gd(el + off[i], 0, Dl, 1, s->A[i].p, 0, (long long)d * Dr, 1, Y.p, 0, (long long)d * Dr, 1, Dl,
                     d * Dr, Dl, 1)));
      if (dens) TRY(rho_partial64(Lc, zp(s->A[i]), zp(Y), Dl, d, Dr, zp(part) + rho_part_count(i, d)));
      TRY(gemm(s, gd(s->A[i].p, 0, 1, Dr, Y.p, 0, Dr, 1, el + off[i + 1], 0, Dr, 1, Dr, Dr, Dl * d, 1, 1)));
    }
    if (dens) TRY(rho_apply64(Lc, zp(part), L, d, zp(opsd), nops, zp(vals)));
    if (s->canonical && !dens) {
      for (int i = 1; i < L; ++i) TRY(eye64(Lc, er + off[i], s->dims[i]));
    }
    for (int i = L - 1; i >= 0 && !s->canonical; --i) {
      const int Dl = s->dims[i], Dr = s->dims[i + 1];
      TRY(mirror_site64(Lc, zp(s->A[i]), zp(s->Atmp), Dl, d, Dr));
      TRY(gemm(s, gd(er + off[i + 1], 0, Dr, 1, s->Atmp.p, 0, (long long)d * Dl, 1, Y.p, 0, (long long)d * Dl, 1,
                     Dr, d * Dl, Dr, 1)));
      TRY(gemm(s, gd(s->Atmp.p, 0, 1, Dl, Y.p, 0, Dl, 1, er + off[i], 0, Dl, 1, Dl, Dl, Dr * d, 1, 1)));
    }
    for (int i = 0; i < L && !dens; ++i) {
      const int Dl = s->dims[i], Dr = s->dims[i + 1];
      for (int k = 0; k < nops; ++k) {
        // OA[a][s][b] = sum_t O[s][t] A[a][t][b]   (batched over a)
        TRY(gemm(s, gd(zp(opsd) + (size_t)k * d * d, 0, d, 1, s->A[i].p, (long long)d * Dr, Dr, 1, OA.p,
                       (long long)d * Dr, Dr, 1, d, Dr, d, Dl)));
        // Z[a][(s b)] = El[i][a][a0] OA[a0][(s b)]
        TRY(gemm(s, gd(el + off[i], 0, Dl, 1, OA.p, 0, (long long)d * Dr, 1, Z.p, 0, (long long)d * Dr, 1, Dl,
                       d * Dr, Dl, 1)));
        // Wm[b][b'] = sum conj(A[(a s)][b]) Z[(a s)][b']
        TRY(gemm(s, gd(s->A[i].p, 0, 1, Dr, Z.p, 0, Dr, 1, Wm.p, 0, Dr, 1, Dr, Dr, Dl * d, 1, 1)));
        TRY(dotu64(Lc, zp(Wm), er + off[i + 1], (size_t)Dr * Dr, zp(vals) + (size_t)k * L + i, static_cast<double*>(s->red.p)));
      }
    }
    std::vector<z64> h((size_t)nops * L), nrm(1);
    TRYCUDA(cudaMemcpyAsync(h.data(), vals.p, sizeof(z64) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    TRYCUDA(cudaMemcpyAsync(nrm.data(), el + off[L], sizeof(z64), cudaMemcpyDeviceToHost, c->stream));
    TRYCUDA(cudaStreamSynchronize(c->stream));
    const double n = nrm[0].x;
    for (size_t j = 0; j < h.size(); ++j) {
      out[2 * j] = h[j].x / n;
      out[2 * j + 1] = h[j].y / n;
    }
    return 0;
  };
  if (!e) e = run();
  cleanup();
  return e;
}

extern "C" int tevo_gemm(tevo_ctx c, int precision, int M, int N, int K, const double* A, const double* B,
                         double* C) {
  if (!c || !A || !B || !C || M < 1 || N < 1 || K < 1) return TEVO_EINVAL;
  const int oz = oz_slices_of(precision);
  if (oz < 0 || (oz && strip_oz(precision) != TEVO_FP64)) return TEVO_EINVAL;
  precision = strip_oz(precision);
  if (precision < TEVO_FP64 || precision > TEVO_BF16X3) return TEVO_EINVAL;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15)
    return TEVO_EINVAL;
  if (precision != TEVO_FP64) return mixed_gemm(c, precision, M, N, K, A, B, C);
  Buf ws;
  GemmDesc g = gd(A, 0, K, 1, B, 0, 1, K, C, 0, N, 1, M, N, K, 1);
  if (oz) {
    // [error flag | slices, exponents, partials]
    int e = dalloc(c, ws, 256 + ozgemm64_workspace(g, oz, c->num_sms));
    int flag = 0;
    if (!e && cudaMemsetAsync(ws.p, 0, sizeof(int), c->stream) != cudaSuccess) e = TEVO_ECUDA;
    if (!e)
      e = ozgemm64(launch_of(c), g, oz, static_cast<char*>(ws.p) + 256, ws.bytes - 256, static_cast<int*>(ws.p));
    if (!e && (cudaMemcpyAsync(&flag, ws.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
               cudaStreamSynchronize(c->stream) != cudaSuccess))
      e = TEVO_ECUDA;
    dfree(c, ws);
    if (!e && flag) e = TEVO_ETIMEOUT;
    return e;
  }
  size_t need = zgemm64_workspace(g, c->num_sms);
  int e = dalloc(c, ws, need);
  if (!e) e = zgemm64(launch_of(c), g, ws.p, ws.bytes);
  if (!e && cudaStreamSynchronize(c->stream) != cudaSuccess) e = TEVO_ECUDA;
  dfree(c, ws);
  return e;
}

extern "C" int tevo_gemm_noalloc(tevo_ctx c, int precision, int M, int N, int K, const double* A, const double* B,
                                 double* C) {
  if (!c || !A || !B || !C || M < 1 || N < 1 || K < 1) return TEVO_EINVAL;
  if (precision < TEVO_FP64 || precision > TEVO_BF16X3) return TEVO_EINVAL;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15)
    return TEVO_EINVAL;
  return noalloc_gemm(launch_of(c), c->device, precision, M, N, K, A, B, C);
}

extern "C" int tevo_wait_selftest(tevo_ctx c, double limit_ms, int* code) {
  if (!c || !code || !(limit_ms > 0) || limit_ms > 5000) return TEVO_EINVAL;
  Buf flag;
  TRY(dalloc(c, flag, 256));
  int e = cudaMemsetAsync(flag.p, 0, sizeof(int), c->stream) == cudaSuccess ? 0 : TEVO_ECUDA;
  if (!e) e = tc_wait_selftest(launch_of(c), static_cast<int*>(flag.p), limit_ms);
  if (!e && (cudaMemcpyAsync(code, flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
             cudaStreamSynchronize(c->stream) != cudaSuccess))
    e = TEVO_ECUDA;
  dfree(c, flag);
  if (e) return e;
  return *code ? TEVO_ETIMEOUT : 0;
}

extern "C" int mps_overlap(tevo_mps a, tevo_mps b, double* log_abs, double* phase) {
  if (!a || !b || !log_abs || !phase) return TEVO_EINVAL;
  if (a->L != b->L || a->d != b->d) return TEVO_ESHAPE;
  tevo_ctx c = b->ctx;
  Launch Lc = launch_of(c);
  const int L = a->L, d = a->d;
  size_t emax = 1, ymax = 1;
  for (int i = 0; i <= L; ++i) emax = std::max(emax, (size_t)a->dims[i] * b->dims[i]);
  for (int i = 0; i < L; ++i) ymax = std::max(ymax, (size_t)a->dims[i] * d * b->dims[i + 1]);
  Buf E0, E1, Y, acc;
  int e = dalloc(c, E0, sizeof(z64) * emax);
  if (!e) e = dalloc(c, E1, sizeof(z64) * emax);
  if (!e) e = dalloc(c, Y, sizeof(z64) * ymax);
  if (!e) e = dalloc(c, acc, sizeof(double) * 4);
  if (!e) e = ensure(c, b->gemm_ws, (size_t)48 << 20);
  if (!e) e = ensure(c, b->red, sizeof(double) * 4096);
  auto run = [&]() -> int {
    double zero[4] = {0, 0, 0, 0};
    TRYCUDA(cudaMemcpyAsync(acc.p, zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    TRY(fill64(Lc, zp(E0), 1, 1.0, 0.0));
    for (int i = 0; i < L; ++i) {
      const int al = a->dims[i], ar = a->dims[i + 1], bl = b->dims[i], br = b->dims[i + 1];
      // Y[a0][(s b)] = E[a0][b0] B[b0][(s b)];  E'[a][b] = sum conj(A[(a0 s)][a]) Y[(a0 s)][b]
      TRY(gemm(b, gd(E0.p, 0, bl, 1, b->A[i].p, 0, (long long)d * br, 1, Y.p, 0, (long long)d * br, 1, al, d * br,
                     bl, 1)));
      TRY(gemm(b, gd(a->A[i].p, 0, 1, ar, Y.p, 0, br, 1, E1.p, 0, br, 1, ar, br, al * d, 1, 1)));
      TRY(rescale64(Lc, zp(E1), (size_t)ar * br, reinterpret_cast<double*>(acc.p), static_cast<double*>(b->red.p)));
      std::swap(E0, E1);
    }
    double h[4];
    z64 z;
    TRYCUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    TRYCUDA(cudaMemcpyAsync(&z, E0.p, sizeof(z64), cudaMemcpyDeviceToHost, c->stream));
    TRYCUDA(cudaStreamSynchronize(c->stream));
    const double az = std::hypot(z.x, z.y);
    *log_abs = az > 0 ? h[0] + std::log(az) : -INFINITY;
    *phase = std::atan2(z.y, z.x);
    return 0;
  };
  if (!e) e = run();
  for (Buf* p : {&E0, &E1, &Y, &acc}) dfree(c, *p);
  return e;
}
