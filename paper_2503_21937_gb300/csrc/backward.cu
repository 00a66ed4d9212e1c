// Reverse-mode gradients of the differentiable semirings.
#include "engine.h"

int backward_impl(lob_engine* e, u32 out_rel, const float* grad_tags, float* const* grad_inputs, int mem) {
  (void)out_rel; (void)grad_tags; (void)grad_inputs; (void)mem;
  if (!e->ran_diff) throw LobError(LOB_E_STATE, "lob_backward needs a completed LOB_DIFF_* run");
  throw LobError(LOB_E_STATE, "backward not available");
}
