// Kernels and launch table for 2 fluid(s), MODE_EXACT (this file is compiled without FMA contraction).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_exact_nf2() { return Launch<2, true>::fns(); }
}  // namespace mfc
