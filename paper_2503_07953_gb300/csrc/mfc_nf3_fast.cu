// Kernels and launch table for 3 fluid(s), MODE_FAST and MODE_MIXED.
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_fast_nf3() { return Launch<3, false>::fns(); }
}  // namespace mfc
