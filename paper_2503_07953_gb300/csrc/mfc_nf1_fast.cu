// Kernels and launch table for 1 fluid(s), MODE_FAST and MODE_MIXED.
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_fast_nf1() { return Launch<1, false>::fns(); }
}  // namespace mfc
