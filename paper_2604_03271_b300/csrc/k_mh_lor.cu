// k_mh_lor.cu -- Lorentzian instantiations of the fused Metropolis kernel.
#include "k_mh_impl.cuh"

namespace smc {
mh_fn mh_pick_lor(int J, int G, int R) { return mh_pick_family<FAM_LORENTZ>(J, G, R); }
}  // namespace smc
