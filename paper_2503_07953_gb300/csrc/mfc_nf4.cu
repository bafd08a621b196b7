// Kernels and launch table for 4 fluid(s).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_nf4() { return Launch<4>::fns(); }
}  // namespace mfc
