// Kernels and launch table for 4 fluid(s), MODE_EXACT (this file is compiled without FMA contraction).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_exact_nf4() { return Launch<4, true>::fns(); }
}  // namespace mfc
