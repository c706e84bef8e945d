// sph_fused_density.cu -- the list-free density pass (density and EOS inside
// the neighbour search, with |N(i)| and n_i), mixed precision and FP64; the
// kernels are in sph_fused.cuh.
#include "sph_fused.cuh"

namespace sphg {

int launch_fused_density(const Launch& L, const NbArgs& a, const PairArgs& pa, int K, int mixed)
{
    if (a.n <= 0 || a.nunits <= 0) return 0;
    if (mixed) {
        SPH_FUSED_DISPATCH(k_fused_density_mixed, K, L, a, pa);
    } else {
        SPH_FUSED_DISPATCH(k_fused_density_fp64, K, L, a, pa);
    }
    return 1;
}

}  // namespace sphg
