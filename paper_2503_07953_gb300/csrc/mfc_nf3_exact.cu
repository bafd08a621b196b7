// Kernels and launch table for 3 fluid(s), MODE_EXACT (this file is compiled without FMA contraction).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_exact_nf3() { return Launch<3, true>::fns(); }
}  // namespace mfc
