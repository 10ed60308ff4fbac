// kern_si4.cu -- single integrator and advection kernels of 4 dimensions
// (dispatched from kern_si.cu).
#include "kern_si_nd.cuh"

namespace odp {

ODP_SI_INSTANTIATE(4)

}  // namespace odp
