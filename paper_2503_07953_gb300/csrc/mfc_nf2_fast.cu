// Kernels and launch table for 2 fluid(s), MODE_FAST and MODE_MIXED.
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_fast_nf2() { return Launch<2, false>::fns(); }
}  // namespace mfc
