// Instantiation of the fused kernels for the sparsely sampled 37 x 37 patch
// (radius 18, every third pixel: 13 x 13 samples), both one-lane tile variants, with
// the window unrolled like the dense radii.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_sparse(int r, int stride) {
    if (r == SPARSE_RADIUS && stride == SPARSE_STRIDE) return make_ops<SPARSE_RADIUS, 0, SPARSE_STRIDE>();
    return nullptr;
}

}  // namespace pcurv
