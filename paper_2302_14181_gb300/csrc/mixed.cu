// Tensor-core (tcgen05) sweep of the low-precision forms.
#include "tevo_mixed.h"

namespace tevo {

struct MixedMPO {};
struct MixedState {};

int mixed_prepare(tevo_ctx, tevo_mpo, tevo_mps, int) { return TEVO_EUNSUPPORTED; }
int mixed_build_right_envs(tevo_ctx, tevo_mpo, tevo_mps, bool, int) { return TEVO_EUNSUPPORTED; }
int mixed_sweep(tevo_ctx, tevo_mpo, tevo_mps, int) { return TEVO_EUNSUPPORTED; }
void mixed_mpo_destroy(tevo_ctx, MixedMPO*& m) { delete m; m = nullptr; }
void mixed_state_destroy(tevo_ctx, MixedState*& m) { delete m; m = nullptr; }

}  // namespace tevo
