// k_mh_gauss.cu -- Gaussian instantiations of the fused Metropolis kernel.
#include "k_mh_impl.cuh"

namespace smc {
mh_fn mh_pick_gauss(int J, int G, int R) { return mh_pick_family<FAM_GAUSS>(J, G, R); }
}  // namespace smc
