// k_mh_pv.cu -- pseudo-Voigt instantiations of the fused Metropolis kernel.
#include "k_mh_impl.cuh"

namespace smc {
mh_fn mh_pick_pv(int J, int G, int R) { return mh_pick_family<FAM_PV>(J, G, R); }
}  // namespace smc
