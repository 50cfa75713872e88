// Second-order (TSC) particle kernel, frozen species, runtime-sized region (see push_impl.cuh).
#include "push_impl.cuh"

namespace gbpic {

cudaError_t launch_push2_frozen_dyn(pic_ctx *c, int si, const ExtDev &ext) { return push::launch_variant<2, true, false>(c, si, ext); }

}  // namespace gbpic
