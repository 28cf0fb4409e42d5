// k_mh_full_pv.cu -- pseudo-Voigt instantiations of the coupled-grid Metropolis kernel.
#include "k_mh_full.cuh"

namespace smc {
mh_fn mhf_pick_pv(int J, int G) { return mhf_pick_family<FAM_PV>(J, G); }
}  // namespace smc
