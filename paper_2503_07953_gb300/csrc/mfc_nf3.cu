// Kernels and launch table for 3 fluid(s).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_nf3() { return Launch<3>::fns(); }
}  // namespace mfc
