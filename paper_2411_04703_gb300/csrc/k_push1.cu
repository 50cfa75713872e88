// First-order (CIC) instantiation of the fused particle kernel (see push_impl.cuh).
#include "push_impl.cuh"

namespace gbpic {

cudaError_t launch_push_order1(pic_ctx *c, int si, const ExtDev &ext) { return push::launch_order<1>(c, si, ext); }

}  // namespace gbpic
