// kern_si6.cu -- single integrator and advection kernels of 6 dimensions
// (dispatched from kern_si.cu).
#include "kern_si_nd.cuh"

namespace odp {

ODP_SI_INSTANTIATE(6)

}  // namespace odp
