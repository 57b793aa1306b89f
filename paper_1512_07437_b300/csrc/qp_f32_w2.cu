// Forms of k_posterior_f32 with 2 warp(s) per pair (see qp_f32.cuh): the two
// occupancy variants, stored and checkpointed, root-mean-square and linear
// combination.
#include "qp_f32.cuh"

namespace qpk {

F32Kernel f32_kernel_w2(int variant, bool ckpt, bool lin) {
    if (lin) {
        if (ckpt) return variant == 1 ? k_posterior_f32_v1<true, 2, true> : k_posterior_f32_v0<true, 2, true>;
        return variant == 1 ? k_posterior_f32_v1<false, 2, true> : k_posterior_f32_v0<false, 2, true>;
    }
    if (ckpt) return variant == 1 ? k_posterior_f32_v1<true, 2, false> : k_posterior_f32_v0<true, 2, false>;
    return variant == 1 ? k_posterior_f32_v1<false, 2, false> : k_posterior_f32_v0<false, 2, false>;
}

}  // namespace qpk
