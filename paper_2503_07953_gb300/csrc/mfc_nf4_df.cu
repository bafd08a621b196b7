// Directional sweeps for 4 fluid(s) in MODE_DF (double-float WENO5).
#include "mfc_launch_impl.cuh"

namespace mfc {
cudaError_t sweep_df_nf4(const Consts& C, int dir, int mode, SweepArgs A, cudaStream_t s) {
    return sweep_df<4>(C, dir, mode, A, s);
}
}  // namespace mfc
