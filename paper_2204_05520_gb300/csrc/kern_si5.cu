// kern_si5.cu -- single integrator and advection kernels of 5 dimensions
// (dispatched from kern_si.cu).
#include "kern_si_nd.cuh"

namespace odp {

ODP_SI_INSTANTIATE(5)

}  // namespace odp
