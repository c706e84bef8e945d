// sph_fused_momentum.cu -- the list-free momentum and energy pass (the pair
// sums inside the neighbour search), mixed precision and FP64; the kernels are in
// sph_fused.cuh.
#include "sph_fused.cuh"

namespace sphg {

int launch_fused_momentum(const Launch& L, const NbArgs& a, const PairArgs& pa, int K, int mixed)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (mixed) {
        SPH_FUSED_DISPATCH(k_fused_momentum_mixed, K, L, a, pa);
    } else {
        SPH_FUSED_DISPATCH(k_fused_momentum_fp64, K, L, a, pa);
    }
    return 1;
}

}  // namespace sphg
