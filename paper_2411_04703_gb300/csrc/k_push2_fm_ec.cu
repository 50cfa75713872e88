// Second-order (TSC) particle kernel, mobile species, compile-time region, energy-conserving gather (see push_impl.cuh).
#include "push_impl.cuh"

namespace gbpic {

cudaError_t launch_push2_mobile_fixed_ec(pic_ctx *c, int si, const ExtDev &ext) { return push::launch_variant<2, false, true, 1>(c, si, ext); }

}  // namespace gbpic
