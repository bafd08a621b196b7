// Kernels and launch table for 1 fluid(s), MODE_EXACT (this file is compiled without FMA contraction).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_exact_nf1() { return Launch<1, true>::fns(); }
}  // namespace mfc
