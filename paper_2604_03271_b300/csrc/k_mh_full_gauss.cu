// k_mh_full_gauss.cu -- Gaussian instantiations of the coupled-grid Metropolis kernel.
#include "k_mh_full.cuh"

namespace smc {
mh_fn mhf_pick_gauss(int J, int G) { return mhf_pick_family<FAM_GAUSS>(J, G); }
}  // namespace smc
