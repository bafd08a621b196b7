// Kernels and launch table for 2 fluid(s).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_nf2() { return Launch<2>::fns(); }
}  // namespace mfc
