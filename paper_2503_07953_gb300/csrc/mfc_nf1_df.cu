// Directional sweeps for 1 fluid(s) in MODE_DF (double-float WENO5).
#include "mfc_launch_impl.cuh"

namespace mfc {
cudaError_t sweep_df_nf1(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s) {
    return sweep_df<1>(C, dir, mode, A, s);
}
}  // namespace mfc
