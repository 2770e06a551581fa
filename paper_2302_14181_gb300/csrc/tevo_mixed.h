// Interface between the sweep driver (api.cu) and the tensor-core sweep (mixed.cu).
#pragma once

#include <vector>

#include "tevo_internal.h"

namespace tevo {

struct MixedMPO;
struct MixedState;

// low-precision copies of the MPO operands and per-state workspace
int mixed_prepare(tevo_ctx c, tevo_mpo W, tevo_mps s, int precision);
// right environments of <bra|W|psi> with tensor-core contractions; bra_fresh
// selects the fitted set (true) or psi itself (false) as the bra
int mixed_build_right_envs(tevo_ctx c, tevo_mpo W, tevo_mps s, bool bra_fresh, int precision);
// one sweep with tensor-core contractions and fp64 QR
int mixed_sweep(tevo_ctx c, tevo_mpo W, tevo_mps s, int precision);
// centre at site 1 with tensor-core contractions (into the fitted set)
int mixed_centre(tevo_ctx c, tevo_mpo W, tevo_mps s, int precision);
// device error flag of the tensor-core kernels (bounded waits); copies it to *flag (async)
int mixed_error_flag(tevo_ctx c, tevo_mps s, int* flag);
// standalone complex GEMM (tevo_gemm)
int mixed_gemm(tevo_ctx c, int precision, int M, int N, int K, const void* A, const void* B, void* C);
// tevo_gemm_noalloc (noalloc.cu)
int noalloc_gemm(const Launch& L, int device, int precision, int M, int N, int K, const void* A, const void* B,
                 void* C);
void mixed_mpo_destroy(tevo_ctx c, MixedMPO*& m);
void mixed_state_destroy(tevo_ctx c, MixedState*& m);

// accessors into the handles (api.cu)
int mps_L(tevo_mps s);
int mps_d(tevo_mps s);
const std::vector<int>& mps_dims(tevo_mps s);
MixedState*& mps_mixed(tevo_mps s);
MixedMPO*& mpo_mixed(tevo_mpo W);
int mpo_wl(tevo_mpo W, int i);
int mpo_wr(tevo_mpo W, int i);
const void* mpo_dev_wr(tevo_mpo W, int i);
const void* mpo_dev_wl(tevo_mpo W, int i);
void* mps_site(tevo_mps s, int i, bool fresh);
void* mps_env_slot(tevo_mps s, int b);
void* mps_buf_T(tevo_mps s);
void* mps_buf_X(tevo_mps s);
void* mps_buf_Bq(tevo_mps s);
void* mps_buf_Atmp(tevo_mps s);
int mps_qr_q(tevo_mps s, int m, int n);
int mps_store_right(tevo_mps s, int i);
int mps_store_left(tevo_mps s, int i);
int ctx_alloc(tevo_ctx c, void** p, size_t bytes);
void ctx_free(tevo_ctx c, void* p);
Launch ctx_launch(tevo_ctx c);

}  // namespace tevo
