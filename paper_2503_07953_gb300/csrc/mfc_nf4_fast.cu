// Kernels and launch table for 4 fluid(s), MODE_FAST and MODE_MIXED.
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_fast_nf4() { return Launch<4, false>::fns(); }
}  // namespace mfc
