// k_mh_phase.cu -- instantiations of the powder-diffraction phase Metropolis kernel.
#include "k_mh_phase.cuh"

namespace smc {
mh_fn mhp_pick(int J, int G) { return mhp_pick_tile(J, G); }
}  // namespace smc
