// Kernels and launch table for 1 fluid(s).
#include "mfc_launch_impl.cuh"

namespace mfc {
const LaunchFns& launch_fns_nf1() { return Launch<1>::fns(); }
}  // namespace mfc
