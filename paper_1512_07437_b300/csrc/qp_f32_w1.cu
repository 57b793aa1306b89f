// Forms of k_posterior_f32 with 1 warp(s) per pair (see qp_f32.cuh): the two
// occupancy variants, stored and checkpointed, root-mean-square and linear
// combination.
#include "qp_f32.cuh"

namespace qpk {

F32Kernel f32_kernel_w1(int variant, bool ckpt, bool lin) {
    if (lin) {
        if (ckpt) return variant == 1 ? k_posterior_f32_v1<true, 1, true> : k_posterior_f32_v0<true, 1, true>;
        return variant == 1 ? k_posterior_f32_v1<false, 1, true> : k_posterior_f32_v0<false, 1, true>;
    }
    if (ckpt) return variant == 1 ? k_posterior_f32_v1<true, 1, false> : k_posterior_f32_v0<true, 1, false>;
    return variant == 1 ? k_posterior_f32_v1<false, 1, false> : k_posterior_f32_v0<false, 1, false>;
}

}  // namespace qpk
