// Directional sweeps for 2 fluid(s) in MODE_DF (double-float WENO5): fused, and split into
// reconstruction and Riemann kernels.
#include "mfc_launch_impl.cuh"

namespace mfc {
cudaError_t sweep_df_nf2(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s) {
    return sweep_df<2>(C, dir, mode, A, s);
}
cudaError_t split_df_nf2(const Consts& C, int dir, int phase, SweepArgs A, SplitChunk K, cudaStream_t s) {
    return split_df<2>(C, dir, phase, A, K, s);
}
}  // namespace mfc
