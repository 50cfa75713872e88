// Second-order (TSC) particle kernel, frozen species, compile-time region (default tile) (see push_impl.cuh).
#include "push_impl.cuh"

namespace gbpic {

cudaError_t launch_push2_frozen_fixed(pic_ctx *c, int si, const ExtDev &ext) { return push::launch_variant<2, true, true>(c, si, ext); }

}  // namespace gbpic
