// k_mh_full_lor.cu -- Lorentzian instantiations of the coupled-grid Metropolis kernel.
#include "k_mh_full.cuh"

namespace smc {
mh_fn mhf_pick_lor(int J, int G) { return mhf_pick_family<FAM_LORENTZ>(J, G); }
}  // namespace smc
